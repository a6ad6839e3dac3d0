// k_device.cuh -- device helpers shared by the evaluation kernels: 3-vectors,
// rigid transforms, the serial-chain forward kinematics (Sec. 3.1), the box
// signed distance, the smoothed collision distance (Eq. 10), the bound cost
// (Eq. 17) and log cosh.  Every function is inline; each translation unit
// that includes this file gets its own copy.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace crgb {
namespace {

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float norm(V3 a) { return sqrtf(dot(a, a)); }

// point x (link frame centre c) through a row-major 3x4 [R|p]
// T: 16-byte aligned 3x4 transform (three float4 rows)
__device__ __forceinline__ V3 tf_point(const float* T, float cx, float cy, float cz) {
  const float4* R = reinterpret_cast<const float4*>(T);
  const float4 a = R[0], b = R[1], c = R[2];
  return v3(fmaf(a.x, cx, fmaf(a.y, cy, fmaf(a.z, cz, a.w))),
            fmaf(b.x, cx, fmaf(b.y, cy, fmaf(b.z, cz, b.w))),
            fmaf(c.x, cx, fmaf(c.y, cy, fmaf(c.z, cz, c.w))));
}

// One joint of a serial chain (Sec. 3.1): N = T F_j J_axis(theta_j), where
// F_j J is the "full link transformation" of App. E.1's joint table (two
// columns of F mixed by cos / sin of theta_j).
__device__ __forceinline__ void fk_joint(const float* F, int ax, float s, float c, const float (&T)[12],
                                         float (&N)[12]) {
  float A[12];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float f0 = F[4 * r], f1 = F[4 * r + 1], f2 = F[4 * r + 2];
    if (ax == 0) {
      A[4 * r] = f0;
      A[4 * r + 1] = fmaf(f1, c, f2 * s);
      A[4 * r + 2] = fmaf(-f1, s, f2 * c);
    } else if (ax == 1) {
      A[4 * r] = fmaf(f0, c, -f2 * s);
      A[4 * r + 1] = f1;
      A[4 * r + 2] = fmaf(f0, s, f2 * c);
    } else {
      A[4 * r] = fmaf(f0, c, f1 * s);
      A[4 * r + 1] = fmaf(-f0, s, f1 * c);
      A[4 * r + 2] = f2;
    }
    A[4 * r + 3] = F[4 * r + 3];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int col = 0; col < 4; ++col) {
      float v = fmaf(T[4 * r], A[col], fmaf(T[4 * r + 1], A[4 + col], T[4 * r + 2] * A[8 + col]));
      N[4 * r + col] = col == 3 ? v + T[4 * r + 3] : v;
    }
  }
}

// Serial chain: T_j = T_{j-1} F_j J_axis(theta_j) from T_{-1} = I.  Writes
// T_0..T_{dof-1} (12 floats each).
__device__ __forceinline__ void fk_chain(const float* fix, const int* axis, int dof,
                                         const float* q, const float2* sc, float* out) {
  float T[12] = {1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f};
  for (int j = 0; j < dof; ++j) {
    float s, c;
    if (sc) {
      s = sc[j].x;
      c = sc[j].y;
    } else {
      sincosf(q[j], &s, &c);
    }
    float N[12];
    fk_joint(fix + 12 * j, axis[j], s, c, T, N);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      T[k] = N[k];
      out[12 * j + k] = N[k];
    }
  }
}

// One row of the serial chain: row r of T_j = (row r of T_{j-1}) F_j J(theta_j)
// depends on row r alone, so three threads can run a chain together.  The
// same operations as fk_joint / fk_chain for that row (bit-identical); writes
// row r of T_0..T_{dof-1} into out (12 floats per joint).
__device__ __forceinline__ void fk_chain_row(const float* fix, const int* axis, int dof, const float2* sc,
                                             int row, float* out) {
  float t0 = row == 0 ? 1.f : 0.f, t1 = row == 1 ? 1.f : 0.f, t2 = row == 2 ? 1.f : 0.f, t3 = 0.f;
  for (int j = 0; j < dof; ++j) {
    const float s = sc[j].x, c = sc[j].y;
    const float* F = fix + 12 * j;
    const int ax = axis[j];
    float A[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float f0 = F[4 * r], f1 = F[4 * r + 1], f2 = F[4 * r + 2];
      if (ax == 0) {
        A[4 * r] = f0;
        A[4 * r + 1] = fmaf(f1, c, f2 * s);
        A[4 * r + 2] = fmaf(-f1, s, f2 * c);
      } else if (ax == 1) {
        A[4 * r] = fmaf(f0, c, -f2 * s);
        A[4 * r + 1] = f1;
        A[4 * r + 2] = fmaf(f0, s, f2 * c);
      } else {
        A[4 * r] = fmaf(f0, c, f1 * s);
        A[4 * r + 1] = fmaf(-f0, s, f1 * c);
        A[4 * r + 2] = f2;
      }
      A[4 * r + 3] = F[4 * r + 3];
    }
    float n[4];
#pragma unroll
    for (int col = 0; col < 4; ++col) {
      const float v = fmaf(t0, A[col], fmaf(t1, A[4 + col], t2 * A[8 + col]));
      n[col] = col == 3 ? v + t3 : v;
    }
    t0 = n[0];
    t1 = n[1];
    t2 = n[2];
    t3 = n[3];
    *reinterpret_cast<float4*>(out + 12 * j + 4 * row) = make_float4(t0, t1, t2, t3);
  }
}

// Box signed distance in the box frame (textbook: Euclidean outside, minus
// the smallest face gap inside) and its gradient in the box frame; inside,
// the face of the largest q wins, lowest axis on ties.
__device__ __forceinline__ float sdf_local(float ux, float uy, float uz, float4 h, V3& gu) {
  float qx = fabsf(ux) - h.x, qy = fabsf(uy) - h.y, qz = fabsf(uz) - h.z;
  float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
  float outside = sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
  int a = 0;
  float mq = qx;
  if (qy > mq) { a = 1; mq = qy; }
  if (qz > mq) { a = 2; mq = qz; }
  float sx = ux >= 0.f ? 1.f : -1.f, sy = uy >= 0.f ? 1.f : -1.f, sz = uz >= 0.f ? 1.f : -1.f;
  if (outside > 0.f) {
    float inv = 1.f / outside;
    gu = v3(sx * mx * inv, sy * my * inv, sz * mz * inv);
  } else {
    gu = v3(a == 0 ? sx : 0.f, a == 1 ? sy : 0.f, a == 2 ? sz : 0.f);
  }
  return outside + fminf(mq, 0.f);
}

// Eq. 10 smoothed collision distance and its slope
__device__ __forceinline__ float smooth_dist(float d, float eta, float inv_eta, float& slope) {
  if (d > 0.f) {
    slope = 1.f;
    return d + 0.5f * eta;
  }
  if (d > -eta) {
    float e = d + eta;
    slope = e * inv_eta;
    return 0.5f * inv_eta * e * e;
  }
  slope = 0.f;
  return 0.f;
}

// Eq. 17 bound cost and slope
__device__ __forceinline__ float bound_cost(float q, float lo, float hi, float e2, float inv_e2,
                                            float& s) {
  if (q < lo) { s = -1.f; return lo - q + 0.5f * e2; }
  if (q < lo + e2) { float d = lo - q + e2; s = -d * inv_e2; return 0.5f * inv_e2 * d * d; }
  if (q > hi) { s = 1.f; return q - hi + 0.5f * e2; }
  if (q > hi - e2) { float d = q - hi + e2; s = d * inv_e2; return 0.5f * inv_e2 * d * d; }
  s = 0.f;
  return 0.f;
}

// log cosh x.  For |x| >= 1/8: |x| + log(1 + e^{-2|x|}) - log 2; below, where
// that form cancels in FP32, the Taylor series x^2/2 - x^4/12 + x^6/45
// (next term 17 x^8 / 2520, below 1e-7 relative there).
__device__ __forceinline__ float logcoshf(float x) {
  const float a = fabsf(x);
  if (a < 0.125f) {
    const float x2 = a * a;
    return x2 * fmaf(x2, fmaf(x2, 1.f / 45.f, -1.f / 12.f), 0.5f);
  }
  return a + log1pf(expf(-2.f * a)) - 0.69314718055994531f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace
}  // namespace crgb
