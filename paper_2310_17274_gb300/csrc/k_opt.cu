// k_opt.cu -- L-BFGS two-loop step, parallel noisy line-search selection and
// best-iterate tracking (Sec. 4.1, Alg. 1, App. A.7), one CTA per seed.
//
// A seed's history (m pairs of n = H*dof floats) is pulled into shared memory
// with one bulk load, so the 2m dependent dot products of the two-loop
// recursion run out of shared memory; the history shift is a relabelling of
// slots while the pairs are written back in newest-last order.
//
// Every dot product is reduced in one fixed order, that of a virtual block of
// 256 threads: element k belongs to virtual thread k mod 256, which adds its
// elements k, k + 256, ... in sequence (fma); lanes of a virtual warp are then
// combined by an xor butterfly and the 8 virtual-warp sums are added in warp
// order.  Seeds of up to 256 variables may run on a single warp (each lane
// playing 8 virtual threads) with bit-identical results, so a seed's result
// never depends on the other seeds of the launch.
#include <cuda_runtime.h>

#include "crgb_internal.cuh"

namespace crgb {

namespace {

constexpr int kVirt = 256;        // virtual threads per seed
constexpr int kSlots = 8;         // element slots per physical thread
constexpr int kMaxN = kVirt * kSlots;

// Partial sums of one dot product for NT physical threads.
template <int NT>
struct Part {
  static constexpr int kP = NT == kVirt ? 1 : kSlots;
  float p[kP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < kP; ++i) p[i] = 0.f;
  }
  // add a*b for element slot e (element k = tid + NT * e)
  __device__ __forceinline__ void fma(int e, float a, float b) {
    if (kP == 1)
      p[0] = fmaf(a, b, p[0]);
    else
      p[e] = fmaf(a, b, p[e]);
  }
};

__device__ __forceinline__ float butterfly(float s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Totals of V dot products; every thread gets them.
template <int NT, int V>
__device__ __forceinline__ void block_sum(Part<NT> (&v)[V], float (&out)[V], float* red) {
  if (NT == kVirt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float s = butterfly(v[k].p[0]);
      if (lane == 0) red[warp * V + k] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float s = 0.f;
      for (int w = 0; w < kVirt / 32; ++w) s += red[w * V + k];
      out[k] = s;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kSlots; ++w) s += butterfly(v[k].p[w]);
      out[k] = s;
    }
  }
}

// NT = 256 for any seed up to 2048 variables; NT = 32 for seeds of at most
// 256 variables (IK), same numerics.
template <int NT>
__global__ void __launch_bounds__(NT) k_opt(const __grid_constant__ OptArgs a) {
  static_assert(NT == 32 || NT == kVirt, "NT");
  extern __shared__ __align__(16) float osm[];
  __shared__ float red[(kVirt / 32) * (CR_MAX_ALPHA + 1)];
  __shared__ float sh_rho[CR_MAX_HISTORY];
  __shared__ float sh_alpha[CR_MAX_HISTORY];

  const int tid = threadIdx.x;
  const int D = a.dof, m = a.prm.history, na = a.prm.n_alpha;
  const cr_opt_state& st = a.st;
  // the evaluation that ran before this launch is complete: its work counter
  // can start over for the next one (saves a memset node per iteration)
  if (a.reset_queue && blockIdx.x == 0 && tid == 0) *a.reset_queue = 0;

  for (int bt = blockIdx.x; bt < a.n_seeds; bt += gridDim.x) {
    // b: the seed's index in the per-seed arrays (the table may list a subset)
    int n, vo, b;
    if (a.seed_tab) {
      const int4 e = a.seed_tab[bt];
      n = e.x;
      vo = e.y;
      b = e.z;
    } else {
      n = a.horizon * D;
      vo = bt * n;
      b = bt;
    }
    float* x = st.x + vo;
    float* g = st.g + vo;
    float* xp = st.x_prev + vo;
    float* gp = st.g_prev + vo;
    float* dir = st.dir + vo;
    float* cand = st.cand + (long long)vo * na;
    float* cgrad = st.cand_grad + (long long)vo * na;
    __syncthreads();

    // ---------------- line-search selection (Alg. 1) ----------------
    if (a.do_select) {
      Part<NT> v[CR_MAX_ALPHA + 1];
#pragma unroll
      for (int l = 0; l <= CR_MAX_ALPHA; ++l) v[l].zero();
#pragma unroll
      for (int e = 0; e < kSlots; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          const float dk = dir[k];
          v[0].fma(e, g[k], dk);
#pragma unroll
          for (int l = 0; l < CR_MAX_ALPHA; ++l)
            if (l < na) v[1 + l].fma(e, cgrad[(long long)l * n + k], dk);
        }
      }
      float tot[CR_MAX_ALPHA + 1];
      block_sum<NT, CR_MAX_ALPHA + 1>(v, tot, red);
      const float c0 = st.c[b];
      const float gd0 = tot[0];
      int idx = 0;
      for (int l = 0; l < na; ++l) {
        const float cl = st.cand_cost[b * na + l];
        bool ok = cl <= c0 + a.prm.armijo_c1 * a.prm.alpha[l] * gd0;
        if (a.prm.flags & CR_WOLFE) {
          const float gld = tot[1 + l];
          if (a.prm.flags & CR_STRONG_WOLFE)
            ok = ok && fabsf(gld) <= a.prm.wolfe_c2 * fabsf(gd0);
          else
            ok = ok && gld >= a.prm.wolfe_c2 * gd0;
        }
        if (ok) idx = l;  // largest passing index; 0 when none passes
      }
      const float cnew = st.cand_cost[b * na + idx];
      const bool better = cnew < st.best_c[b];  // NaN never improves the best
#pragma unroll
      for (int e = 0; e < kSlots; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          const float xv = cand[(long long)idx * n + k];
          x[k] = xv;
          g[k] = cgrad[(long long)idx * n + k];
          if (better) st.best_x[vo + k] = xv;
        }
      }
      __syncthreads();  // every thread has read c[b] and best_c[b]
      if (tid == 0) {
        st.c[b] = cnew;
        st.ls_index[b] = idx;
        if (better) {
          st.best_c[b] = cnew;
          st.best_cfree[b] = st.cand_cfree[b * na + idx];
        }
      }
    }
    if (a.init_best) {
      for (int k = tid; k < n; k += NT) st.best_x[vo + k] = x[k];
      if (tid == 0) st.best_c[b] = st.c[b];
    }

    // ---------------- L-BFGS step (App. A.7) ----------------
    if (a.do_propose) {
      float* hs = osm;                  // [m][n] s pairs, physical slots
      float* hy = osm + (size_t)m * n;  // [m][n]
      float* s_g = st.s + (long long)vo * m;
      float* y_g = st.y + (long long)vo * m;
      float* rho_g = st.rho + b * m;
      for (int k = tid; k < m * n; k += NT) {
        hs[k] = s_g[k];
        hy[k] = y_g[k];
      }
      if (tid < m) sh_rho[tid] = rho_g[tid];
      const int it = st.iter[b];
      float xr[kSlots], gr[kSlots];
#pragma unroll
      for (int e = 0; e < kSlots; ++e) {
        const int k = tid + NT * e;
        xr[e] = k < n ? x[k] : 0.f;
        gr[e] = k < n ? g[k] : 0.f;
      }
      __syncthreads();
      int shift = 0;  // logical pair i (0 = oldest) lives in physical slot (i + shift) % m
      if (it > 0) {
        // the newest pair overwrites the oldest slot (physical 0)
        float sv[kSlots], yv[kSlots];
        Part<NT> ys[1];
        ys[0].zero();
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          sv[e] = k < n ? xr[e] - xp[k] : 0.f;
          yv[e] = k < n ? gr[e] - gp[k] : 0.f;
          if (k < n) ys[0].fma(e, yv[e], sv[e]);
        }
        float yst[1];
        block_sum<NT, 1>(ys, yst, red);
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          if (k < n) {
            hs[k] = sv[e];
            hy[k] = yv[e];
          }
        }
        if (tid == 0) sh_rho[0] = yst[0] > 1e-8f ? 1.f / yst[0] : 0.f;
        shift = 1;
        __syncthreads();
        // write back newest-last
        for (int i = 0; i < m; ++i) {
          const int p = (i + shift) % m;
          for (int k = tid; k < n; k += NT) {
            s_g[(long long)i * n + k] = hs[(long long)p * n + k];
            y_g[(long long)i * n + k] = hy[(long long)p * n + k];
          }
        }
        if (tid < m) rho_g[tid] = sh_rho[(tid + shift) % m];
      }
      for (int k = tid; k < n; k += NT) {
        xp[k] = x[k];
        gp[k] = g[k];
      }
      if (tid == 0) st.iter[b] = it + 1;

      // two-loop recursion: q = g; newest to oldest
      float q[kSlots];
#pragma unroll
      for (int e = 0; e < kSlots; ++e) q[e] = gr[e];
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        const float rho = sh_rho[p];
        if (rho == 0.f) {  // inert pair: alpha = 0, q unchanged
          if (tid == 0) sh_alpha[i] = 0.f;
          continue;
        }
        Part<NT> d[1];
        d[0].zero();
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          if (k < n) d[0].fma(e, hs[(long long)p * n + k], q[e]);
        }
        float dt[1];
        block_sum<NT, 1>(d, dt, red);
        const float al = rho * dt[0];
        if (tid == 0) sh_alpha[i] = al;
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          if (k < n) q[e] = fmaf(-al, hy[(long long)p * n + k], q[e]);
        }
      }
      // H0 = gamma I from the newest valid pair
      float gamma = 1.f;
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        if (sh_rho[p] > 0.f) {
          Part<NT> d[2];
          d[0].zero();
          d[1].zero();
#pragma unroll
          for (int e = 0; e < kSlots; ++e) {
            const int k = tid + NT * e;
            if (k < n) {
              const float sv = hs[(long long)p * n + k], yv = hy[(long long)p * n + k];
              d[0].fma(e, sv, yv);
              d[1].fma(e, yv, yv);
            }
          }
          float dt[2];
          block_sum<NT, 2>(d, dt, red);
          gamma = dt[0] / dt[1];
          break;
        }
      }
#pragma unroll
      for (int e = 0; e < kSlots; ++e) q[e] *= gamma;
      __syncthreads();  // sh_alpha visible
      for (int i = 0; i < m; ++i) {
        const int p = (i + shift) % m;
        const float rho = sh_rho[p];
        if (rho == 0.f) continue;
        Part<NT> d[1];
        d[0].zero();
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          if (k < n) d[0].fma(e, hy[(long long)p * n + k], q[e]);
        }
        float dt[1];
        block_sum<NT, 1>(d, dt, red);
        const float coef = sh_alpha[i] - rho * dt[0];
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          const int k = tid + NT * e;
          if (k < n) q[e] = fmaf(hs[(long long)p * n + k], coef, q[e]);
        }
      }
      // direction and the clipped candidates of Alg. 1
#pragma unroll
      for (int e = 0; e < kSlots; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          const float dk = -q[e];
          dir[k] = dk;
          const int j = k % D;
          const float lo = a.q_lo[j], hi = a.q_hi[j];
          for (int l = 0; l < na; ++l) {
            float v = fmaf(a.prm.alpha[l], dk, xr[e]);
            v = fminf(fmaxf(v, lo), hi);
            cand[(long long)l * n + k] = v;
          }
        }
      }
    }
  }
}

// The largest dynamic shared memory any launch may ask for is set once per
// kernel and device (never lowered), so launches captured in a graph stay
// valid whatever is launched later.
template <int NT>
cudaError_t allow_opt_smem() {
  static unsigned done = 0;  // bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  if (done & bit) return cudaSuccess;
  // 200 KB covers every accepted history * horizon * dof and stays below the
  // opt-in limit together with the kernel's static shared memory
  cudaError_t e = cudaFuncSetAttribute(k_opt<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) done |= bit;
  return e;
}

}  // namespace

int opt_smem_bytes(int history, int n_max) { return 2 * history * n_max * (int)sizeof(float); }

cudaError_t launch_opt(const OptArgs& a, int n_max, cudaStream_t stream) {
  if (a.n_seeds <= 0) return cudaSuccess;
  if (n_max > kMaxN) return cudaErrorInvalidValue;
  const int smem = a.do_propose ? opt_smem_bytes(a.prm.history, n_max) : 0;
  if (n_max <= kVirt) {
    cudaError_t e = allow_opt_smem<32>();
    if (e != cudaSuccess) return e;
    k_opt<32><<<a.n_seeds, 32, smem, stream>>>(a);
  } else {
    cudaError_t e = allow_opt_smem<kVirt>();
    if (e != cudaSuccess) return e;
    k_opt<kVirt><<<a.n_seeds, kVirt, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace crgb
