// k_time.cuh -- device arithmetic of App. "Time-step Discretization" (the
// retiming of Alg. "Time Discretization") and of App. "Solver details" (the
// score that chooses among a solve's seeds), shared by the retiming, the
// seed-choice and the time-discretised solve kernels.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "crgb_internal.cuh"
#include "k_device.cuh"

namespace crgb {
namespace {

// Padded sequence of App. A.5 for one trajectory th [H][D] from q0: three
// copies of q0, theta_1..theta_H, two copies of theta_H.
__device__ __forceinline__ float time_ext(const float* th, const float* q0, int H, int D, int n, int j) {
  if (n <= 2) return q0[j];
  if (n >= H + 2) return th[(H - 1) * D + j];
  return th[(n - 3) * D + j];
}

// Retiming: the App. A.5 stencils scale as 1/dt, 1/dt^2, 1/dt^3, so from the
// stencils at dt = 1 the smallest dt that keeps a sample within the limits
// is the largest of |v1|/v_max, sqrt(|a1|/a_max), cbrt(|j1|/j_max).  This is
// the maximum over the samples k = k0, k0 + stride, ... of the (H + 1) x D
// (sample, joint) pairs; a maximum, so any split of the samples gives the
// same value.  lim: [5][D] q_lo, q_hi, v_max, a_max, j_max.
__device__ __forceinline__ float retime_part(const float* th, const float* q0, const float* lim, int H, int D,
                                             int k0, int stride) {
  float dt = 0.f;
  for (int k = k0; k < (H + 1) * D; k += stride) {
    const int e = k / D + 2, j = k % D;
    const float qm2 = time_ext(th, q0, H, D, e - 2, j), qm1 = time_ext(th, q0, H, D, e - 1, j),
                q00 = time_ext(th, q0, H, D, e, j), qp1 = time_ext(th, q0, H, D, e + 1, j),
                qp2 = time_ext(th, q0, H, D, e + 2, j);
    const float v = (qm2 - 8.f * qm1 + 8.f * qp1 - qp2) * (1.f / 12.f);
    const float a = (-qm2 + 16.f * qm1 - 30.f * q00 + 16.f * qp1 - qp2) * (1.f / 12.f);
    const float jr = (-qm2 + 2.f * qm1 - 2.f * qp1 + qp2) * 0.5f;
    const float vm = lim[2 * D + j], am = lim[3 * D + j], jm = lim[4 * D + j];
    dt = fmaxf(dt, fabsf(v) / vm);
    dt = fmaxf(dt, sqrtf(fabsf(a) / am));
    dt = fmaxf(dt, cbrtf(fabsf(jr) / jm));
  }
  return dt;
}

struct RankWeights {
  float pose, jerk, time, dist;
};

// Score of one seed (App. "Solver details", reading of the unstated blend):
// e_pose = |p - p_g| + d_q at the last state (d_q of Eq. 14 from the trace);
// IK: w_pose e_pose + w_dist |theta_H - q_start|; otherwise w_pose e_pose +
// w_jerk max |jerk| + w_time H dt_b, the jerk of App. A.5's five-point
// stencil at the seed's time step dt_b over every sample and joint.
// fix: [(D+1)][12] fixed transforms, axis: [D], both in shared memory.
__device__ __forceinline__ float seed_score(const float* fix, const int* axis, int D, const ProblemView& pv,
                                            const float* th, float dtb, int ik, RankWeights w) {
  const int H = pv.horizon;
  const float* last = th + (H - 1) * D;
  // end effector of the last state: T_{dof-1} F_ee
  float T[12] = {1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f};
  for (int l = 0; l < D; ++l) {
    float sn, cs;
    sincosf(last[l], &sn, &cs);
    float N[12];
    fk_joint(fix + 12 * l, axis[l], sn, cs, T, N);
#pragma unroll
    for (int k = 0; k < 12; ++k) T[k] = N[k];
  }
  const float* Fe = fix + D * 12;
  float E[12];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float v = fmaf(T[4 * r], Fe[c], fmaf(T[4 * r + 1], Fe[4 + c], T[4 * r + 2] * Fe[8 + c]));
      E[4 * r + c] = c == 3 ? v + T[4 * r + 3] : v;
    }
  const V3 e = v3(E[3] - pv.goal_p[0], E[7] - pv.goal_p[1], E[11] - pv.goal_p[2]);
  float tr = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) tr = fmaf(pv.goal_R[a * 3 + c], E[a * 4 + c], tr);
  float s = w.pose * (norm(e) + (3.f - tr) * 0.25f);
  if (ik) {
    float d2 = 0.f;
    for (int j = 0; j < D; ++j) {
      const float d = last[j] - pv.q_start[j];
      d2 = fmaf(d, d, d2);
    }
    s += w.dist * sqrtf(d2);
  } else {
    float jm = 0.f;
    for (int e2 = 2; e2 <= H + 2; ++e2)
      for (int j = 0; j < D; ++j) {
        const float jr = (-time_ext(th, pv.q_start, H, D, e2 - 2, j) + 2.f * time_ext(th, pv.q_start, H, D, e2 - 1, j) -
                          2.f * time_ext(th, pv.q_start, H, D, e2 + 1, j) + time_ext(th, pv.q_start, H, D, e2 + 2, j)) *
                         0.5f;
        jm = fmaxf(jm, fabsf(jr));
      }
    s += w.jerk * (jm / (dtb * dtb * dtb)) + w.time * (float)H * dtb;
  }
  return s;
}

// Order-free choice: the lower score wins, the lower index on ties; a NaN
// score never wins; bi < 0 means none yet.
__device__ __forceinline__ bool score_better(float s, int i, float bs, int bi) {
  return !isnan(s) && (bi < 0 || s < bs || (s == bs && i < bi));
}

}  // namespace
}  // namespace crgb
