// k_opt.cu -- L-BFGS two-loop step, parallel noisy line-search selection and
// best-iterate tracking (Sec. 4.1, Alg. 1, App. A.7), one CTA per seed.
//
// A seed's history (m pairs of n = H*dof floats) is pulled into shared memory
// with one bulk load, so the 2m dependent dot products of the two-loop
// recursion run out of shared memory; the history shift is a relabelling of
// slots while the pairs are written back in newest-last order.  Every dot
// product is a fixed-shape block reduction (lane sums, xor butterfly, warp
// partials summed in warp order), so the result does not depend on timing.
#include <cuda_runtime.h>

#include "crgb_internal.cuh"

namespace crgb {

namespace {

constexpr int kMaxPerThread = 8;  // n <= 8 * threads variables per seed

// Sum V values over the block of NT threads; every thread gets the totals.
template <int NT, int V>
__device__ __forceinline__ void block_sum(float (&v)[V], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[k] = s;
    if (NT > 32 && lane == 0) red[warp * V + k] = s;
  }
  if (NT > 32) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float s = 0.f;
      for (int w = 0; w < NT / 32; ++w) s += red[w * V + k];
      v[k] = s;
    }
    __syncthreads();
  }
}

// NT threads per seed: 32 for short seeds (IK, n <= 256), 256 otherwise.
template <int NT>
__global__ void __launch_bounds__(NT) k_opt(const __grid_constant__ OptArgs a) {
  constexpr int kOptThreads = NT;
  extern __shared__ __align__(16) float osm[];
  __shared__ float red[(NT / 32) * (CR_MAX_ALPHA + 1)];
  __shared__ float sh_rho[CR_MAX_HISTORY];
  __shared__ float sh_alpha[CR_MAX_HISTORY];

  const int tid = threadIdx.x;
  const int D = a.dof, m = a.prm.history, na = a.prm.n_alpha;
  const cr_opt_state& st = a.st;

  for (int b = blockIdx.x; b < a.n_seeds; b += gridDim.x) {
    int n, vo;
    if (a.seed_tab) {
      const int4 e = a.seed_tab[b];
      n = e.x;
      vo = e.y;
    } else {
      n = a.horizon * D;
      vo = b * n;
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
      float v[CR_MAX_ALPHA + 1];
#pragma unroll
      for (int l = 0; l <= CR_MAX_ALPHA; ++l) v[l] = 0.f;
      for (int k = tid; k < n; k += kOptThreads) {
        const float dk = dir[k];
        v[0] = fmaf(g[k], dk, v[0]);
#pragma unroll
        for (int l = 0; l < CR_MAX_ALPHA; ++l)
          if (l < na) v[1 + l] = fmaf(cgrad[(long long)l * n + k], dk, v[1 + l]);
      }
      block_sum<NT, CR_MAX_ALPHA + 1>(v, red);
      const float c0 = st.c[b];
      const float gd0 = v[0];
      int idx = 0;
      for (int l = 0; l < na; ++l) {
        const float cl = st.cand_cost[b * na + l];
        bool ok = cl <= c0 + a.prm.armijo_c1 * a.prm.alpha[l] * gd0;
        if (a.prm.flags & CR_WOLFE) {
          const float gld = v[1 + l];
          if (a.prm.flags & CR_STRONG_WOLFE)
            ok = ok && fabsf(gld) <= a.prm.wolfe_c2 * fabsf(gd0);
          else
            ok = ok && gld >= a.prm.wolfe_c2 * gd0;
        }
        if (ok) idx = l;  // largest passing index; 0 when none passes
      }
      const float cnew = st.cand_cost[b * na + idx];
      const bool better = cnew < st.best_c[b];  // NaN never improves the best
      for (int k = tid; k < n; k += kOptThreads) {
        const float xv = cand[(long long)idx * n + k];
        x[k] = xv;
        g[k] = cgrad[(long long)idx * n + k];
        if (better) st.best_x[vo + k] = xv;
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
      for (int k = tid; k < n; k += kOptThreads) st.best_x[vo + k] = x[k];
      if (tid == 0) st.best_c[b] = st.c[b];
    }

    // ---------------- L-BFGS step (App. A.7) ----------------
    if (a.do_propose) {
      float* hs = osm;                 // [m][n] s pairs, physical slots
      float* hy = osm + (size_t)m * n; // [m][n]
      float* s_g = st.s + (long long)vo * m;
      float* y_g = st.y + (long long)vo * m;
      float* rho_g = st.rho + b * m;
      for (int k = tid; k < m * n; k += kOptThreads) {
        hs[k] = s_g[k];
        hy[k] = y_g[k];
      }
      if (tid < m) sh_rho[tid] = rho_g[tid];
      const int it = st.iter[b];
      float xr[kMaxPerThread], gr[kMaxPerThread];
#pragma unroll
      for (int u = 0; u < kMaxPerThread; ++u) {
        const int k = tid + u * kOptThreads;
        xr[u] = k < n ? x[k] : 0.f;
        gr[u] = k < n ? g[k] : 0.f;
      }
      __syncthreads();
      int shift = 0;  // logical pair i (0 = oldest) lives in physical slot (i + shift) % m
      if (it > 0) {
        // the newest pair overwrites the oldest slot (physical 0)
        float sv[kMaxPerThread], yv[kMaxPerThread];
        float ys[1] = {0.f};
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          sv[u] = k < n ? xr[u] - xp[k] : 0.f;
          yv[u] = k < n ? gr[u] - gp[k] : 0.f;
          ys[0] = fmaf(yv[u], sv[u], ys[0]);
        }
        block_sum<NT, 1>(ys, red);
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          if (k < n) {
            hs[k] = sv[u];
            hy[k] = yv[u];
          }
        }
        if (tid == 0) sh_rho[0] = ys[0] > 1e-8f ? 1.f / ys[0] : 0.f;
        shift = 1;
        __syncthreads();
        // write back newest-last
        for (int i = 0; i < m; ++i) {
          const int p = (i + shift) % m;
          for (int k = tid; k < n; k += kOptThreads) {
            s_g[(long long)i * n + k] = hs[(long long)p * n + k];
            y_g[(long long)i * n + k] = hy[(long long)p * n + k];
          }
        }
        if (tid < m) rho_g[tid] = sh_rho[(tid + shift) % m];
      }
      for (int k = tid; k < n; k += kOptThreads) {
        xp[k] = x[k];
        gp[k] = g[k];
      }
      if (tid == 0) st.iter[b] = it + 1;

      // two-loop recursion: q = g; newest to oldest
      float q[kMaxPerThread];
#pragma unroll
      for (int u = 0; u < kMaxPerThread; ++u) q[u] = gr[u];
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        const float rho = sh_rho[p];
        if (rho == 0.f) {  // inert pair: alpha = 0, q unchanged
          if (tid == 0) sh_alpha[i] = 0.f;
          continue;
        }
        float d[1] = {0.f};
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          if (k < n) d[0] = fmaf(hs[(long long)p * n + k], q[u], d[0]);
        }
        block_sum<NT, 1>(d, red);
        const float al = rho * d[0];
        if (tid == 0) sh_alpha[i] = al;
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          if (k < n) q[u] = fmaf(-al, hy[(long long)p * n + k], q[u]);
        }
      }
      // H0 = gamma I from the newest valid pair
      float gamma = 1.f;
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        if (sh_rho[p] > 0.f) {
          float d[2] = {0.f, 0.f};
#pragma unroll
          for (int u = 0; u < kMaxPerThread; ++u) {
            const int k = tid + u * kOptThreads;
            if (k < n) {
              const float sv = hs[(long long)p * n + k], yv = hy[(long long)p * n + k];
              d[0] = fmaf(sv, yv, d[0]);
              d[1] = fmaf(yv, yv, d[1]);
            }
          }
          block_sum<NT, 2>(d, red);
          gamma = d[0] / d[1];
          break;
        }
      }
#pragma unroll
      for (int u = 0; u < kMaxPerThread; ++u) q[u] *= gamma;
      __syncthreads();  // sh_alpha visible
      for (int i = 0; i < m; ++i) {
        const int p = (i + shift) % m;
        const float rho = sh_rho[p];
        if (rho == 0.f) continue;
        float d[1] = {0.f};
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          if (k < n) d[0] = fmaf(hy[(long long)p * n + k], q[u], d[0]);
        }
        block_sum<NT, 1>(d, red);
        const float coef = sh_alpha[i] - rho * d[0];
#pragma unroll
        for (int u = 0; u < kMaxPerThread; ++u) {
          const int k = tid + u * kOptThreads;
          if (k < n) q[u] = fmaf(hs[(long long)p * n + k], coef, q[u]);
        }
      }
      // direction and the clipped candidates of Alg. 1
#pragma unroll
      for (int u = 0; u < kMaxPerThread; ++u) {
        const int k = tid + u * kOptThreads;
        if (k < n) {
          const float dk = -q[u];
          dir[k] = dk;
          const int j = k % D;
          const float lo = a.q_lo[j], hi = a.q_hi[j];
          for (int l = 0; l < na; ++l) {
            float v = fmaf(a.prm.alpha[l], dk, xr[u]);
            v = fminf(fmaxf(v, lo), hi);
            cand[(long long)l * n + k] = v;
          }
        }
      }
    }
  }
}

}  // namespace

int opt_smem_bytes(int history, int n_max) { return 2 * history * n_max * (int)sizeof(float); }

cudaError_t launch_opt(const OptArgs& a, int n_max, cudaStream_t stream) {
  if (a.n_seeds <= 0) return cudaSuccess;
  const int smem = a.do_propose ? opt_smem_bytes(a.prm.history, n_max) : 0;
  if (n_max <= 32 * kMaxPerThread) {
    cudaError_t e = cudaFuncSetAttribute(k_opt<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_opt<32><<<a.n_seeds, 32, smem, stream>>>(a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_opt<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_opt<256><<<a.n_seeds, 256, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace crgb
