// k_opt.cu -- L-BFGS two-loop step, parallel noisy line-search selection and
// best-iterate tracking (Sec. 4.1, Alg. 1, App. A.7), one CTA per seed.
//
// A seed's history (m pairs of n = H*dof floats) is a ring of m slots in
// device memory: the pair appended when iter = k > 0 goes to slot (k-1) mod m,
// so an iteration writes one pair and never moves the others.  The ring is
// pulled into shared memory (all loads in flight at once) and the 2m
// dependent dot products of the two-loop recursion run out of shared memory.
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
constexpr int kSlots = 8;         // most element slots per physical thread
constexpr int kMaxN = kVirt * kSlots;
constexpr int kLaneSeedsFrom = 4096;  // seeds of <= 32 variables: one thread each from this many

// Partial sums of one dot product for NT physical threads holding SLOTS
// element slots each (element k = tid + NT * e).  With NT = 256 every slot of
// a thread belongs to the same virtual thread; with NT = 32 slot e is virtual
// thread tid + 32 e.
template <int NT, int SLOTS>
struct Part {
  static constexpr int kP = NT == kVirt ? 1 : SLOTS;
  float p[kP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < kP; ++i) p[i] = 0.f;
  }
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

constexpr int kRed = (kVirt / 32) * (CR_MAX_ALPHA + 1);  // one reduction buffer

// Totals of V dot products; every thread gets them.  Successive calls
// alternate between two buffers (`phase`), so one barrier per call suffices:
// a buffer is rewritten only after the barrier of the call in between, which
// every thread reaches after its reads of the buffer.  Virtual warps with no
// elements add +0 in both forms, so NT = 32 and NT = 256 agree bit for bit.
template <int NT, int SLOTS, int V>
__device__ __forceinline__ void block_sum(Part<NT, SLOTS> (&v)[V], float (&out)[V], float* red2,
                                          int& phase) {
  if (NT == kVirt) {
    float* red = red2 + phase * kRed;
    phase ^= 1;
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
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < SLOTS; ++w) s += butterfly(v[k].p[w]);
      for (int w = SLOTS; w < kVirt / 32; ++w) s += 0.f;
      out[k] = s;
    }
  }
}

__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// One CTA per seed; NT = 256 for seeds of 257..2048 variables, NT = 32 for
// seeds of at most 256 (same numerics); SLOTS = ceil(n_max / NT).
template <int NT, int SLOTS>
__global__ void __launch_bounds__(NT) k_opt(const __grid_constant__ OptArgs a) {
  static_assert(NT == 32 || NT == kVirt, "NT");
  static_assert(NT * SLOTS <= kMaxN && (NT == 32 ? SLOTS <= kSlots : true), "SLOTS");
  // line-search candidates and their gradients stay in registers when few
  constexpr bool kHold = SLOTS <= 2;
  constexpr int kHA = kHold ? CR_MAX_ALPHA : 1;
  extern __shared__ __align__(16) float osm[];
  __shared__ float red[2 * kRed];
  __shared__ float sh_rho[CR_MAX_HISTORY];
  __shared__ float sh_alpha[CR_MAX_HISTORY];
  __shared__ int sh_vp[CR_MAX_HISTORY];    // slots of the pairs with rho != 0, newest first
  __shared__ float sh_vr[CR_MAX_HISTORY];  // and their rho
  __shared__ int sh_nv;
  int phase = 0;

  const int tid = threadIdx.x;
  const int D = a.dof, m = a.prm.history, na = a.prm.n_alpha;
  const cr_opt_state& st = a.st;
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
    float* hs = osm;                  // [m][n] s ring, slots as in device memory
    float* hy = osm + (size_t)m * n;  // [m][n]
    float* s_g = st.s + (long long)vo * m;
    float* y_g = st.y + (long long)vo * m;
    float* rho_g = st.rho + b * m;
    __syncthreads();  // the previous seed is done with shared memory

    // ---- every load that does not depend on the line-search choice, all in
    // flight together: the history ring straight into shared memory, the
    // iterate, previous iterate, direction and candidates; before the
    // previous grid has finished only when that grid cannot have written them
    const bool early = a.early_loads && a.do_select;
    if (!early) pdl_wait();
    if (a.do_propose) {
      const int mn = m * n;
      for (int k = tid; k < mn; k += NT) {
        cp_async4(hs + k, s_g + k);
        cp_async4(hy + k, y_g + k);
      }
      if (tid < m) sh_rho[tid] = rho_g[tid];
    }
    float xr[SLOTS], gr[SLOTS], dr[SLOTS], xpr[SLOTS], gpr[SLOTS], lo[SLOTS], hi[SLOTS];
    float hc[kHA][SLOTS], hg[kHA][SLOTS];
    const int it = a.do_propose ? st.iter[b] : 0;
    const float c_cur = a.do_select ? st.c[b] : 0.f;
    const float c_best = a.do_select ? st.best_c[b] : 0.f;
#pragma unroll
    for (int e = 0; e < SLOTS; ++e) {
      const int k = tid + NT * e;
      const bool ok = k < n;
      lo[e] = ok && a.do_propose ? a.q_lo[k % D] : 0.f;
      hi[e] = ok && a.do_propose ? a.q_hi[k % D] : 0.f;
      xr[e] = ok ? x[k] : 0.f;
      gr[e] = ok ? g[k] : 0.f;
      dr[e] = ok && a.do_select ? dir[k] : 0.f;
      xpr[e] = ok && a.do_propose ? xp[k] : 0.f;
      gpr[e] = ok && a.do_propose ? gp[k] : 0.f;
      if (kHold && a.do_select) {
#pragma unroll
        for (int l = 0; l < kHA; ++l) hc[l][e] = ok && l < na ? cand[(long long)l * n + k] : 0.f;
      }
    }
    // the evaluation's own outputs are read only after it is done
    if (early) pdl_wait();
    if (bt == blockIdx.x) {
      pdl_launch_dependents();
      // the evaluation that ran before this launch is complete: its work
      // counter can start over for the next one (saves a memset node)
      if (a.reset_queue && blockIdx.x == 0 && tid == 0) *a.reset_queue = 0;
    }
    if (kHold && a.do_select) {
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
#pragma unroll
        for (int l = 0; l < kHA; ++l) hg[l][e] = k < n && l < na ? cgrad[(long long)l * n + k] : 0.f;
      }
    }
    float ccost[CR_MAX_ALPHA];  // candidate costs, every thread (same addresses)
#pragma unroll
    for (int l = 0; l < CR_MAX_ALPHA; ++l) ccost[l] = a.do_select && l < na ? st.cand_cost[b * na + l] : 0.f;

    // ---------------- line-search selection (Alg. 1) ----------------
    if (a.do_select) {
      Part<NT, SLOTS> v[CR_MAX_ALPHA + 1];
#pragma unroll
      for (int l = 0; l <= CR_MAX_ALPHA; ++l) v[l].zero();
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          v[0].fma(e, gr[e], dr[e]);
#pragma unroll
          for (int l = 0; l < CR_MAX_ALPHA; ++l)
            if (l < na) v[1 + l].fma(e, kHold ? hg[kHold ? l : 0][e] : cgrad[(long long)l * n + k], dr[e]);
        }
      }
      float tot[CR_MAX_ALPHA + 1];
      // only the first n_alpha + 1 sums are used: reduce 5 or 9 of them when
      // that is enough (the sums themselves do not depend on how many)
      if (na <= 4) {
        block_sum<NT, SLOTS, 5>(reinterpret_cast<Part<NT, SLOTS>(&)[5]>(v),
                                reinterpret_cast<float(&)[5]>(tot), red, phase);
      } else if (na <= 8) {
        block_sum<NT, SLOTS, 9>(reinterpret_cast<Part<NT, SLOTS>(&)[9]>(v),
                                reinterpret_cast<float(&)[9]>(tot), red, phase);
      } else {
        block_sum<NT, SLOTS, CR_MAX_ALPHA + 1>(v, tot, red, phase);
      }
      const float c0 = c_cur;
      const float gd0 = tot[0];
      int idx = 0;
      float cnew = ccost[0];
#pragma unroll
      for (int l = 0; l < CR_MAX_ALPHA; ++l) {
        if (l >= na) break;
        const float cl = ccost[l];
        bool ok = cl <= c0 + a.prm.armijo_c1 * a.prm.alpha[l] * gd0;
        if (a.prm.flags & CR_WOLFE) {
          const float gld = tot[1 + l];
          if (a.prm.flags & CR_STRONG_WOLFE)
            ok = ok && fabsf(gld) <= a.prm.wolfe_c2 * fabsf(gd0);
          else
            ok = ok && gld >= a.prm.wolfe_c2 * gd0;
        }
        if (ok) {  // largest passing index; 0 when none passes
          idx = l;
          cnew = cl;
        }
      }
      const bool better = cnew < c_best;  // NaN never improves the best
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          float xv, gv;
          if (kHold) {
            xv = hc[0][e];
            gv = hg[0][e];
#pragma unroll
            for (int l = 1; l < kHA; ++l)
              if (l == idx) {
                xv = hc[l][e];
                gv = hg[l][e];
              }
          } else {
            xv = cand[(long long)idx * n + k];
            gv = cgrad[(long long)idx * n + k];
          }
          xr[e] = xv;
          gr[e] = gv;
          x[k] = xv;
          g[k] = gv;
          if (better) st.best_x[vo + k] = xv;
        }
      }
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
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
        if (k < n) st.best_x[vo + k] = xr[e];
      }
      if (tid == 0) st.best_c[b] = st.c[b];
    }

    // ---------------- L-BFGS step (App. A.7) ----------------
    if (a.do_propose) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();  // the ring and rho are in shared memory
      // logical pair i (0 = oldest) lives in slot (i + shift) % m; with
      // it > 0 this call appends pair number it, in slot (it - 1) % m
      int shift = 0;
      if (it > 0) {
        const int w = (it - 1) % m;
        float sv[SLOTS], yv[SLOTS];
        Part<NT, SLOTS> ys[1];
        ys[0].zero();
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          sv[e] = k < n ? xr[e] - xpr[e] : 0.f;
          yv[e] = k < n ? gr[e] - gpr[e] : 0.f;
          if (k < n) ys[0].fma(e, yv[e], sv[e]);
        }
        float yst[1];
        block_sum<NT, SLOTS, 1>(ys, yst, red, phase);
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) {
            hs[(long long)w * n + k] = sv[e];
            hy[(long long)w * n + k] = yv[e];
            s_g[(long long)w * n + k] = sv[e];
            y_g[(long long)w * n + k] = yv[e];
          }
        }
        if (tid == 0) {
          const float r = yst[0] > 1e-8f ? 1.f / yst[0] : 0.f;
          sh_rho[w] = r;
          rho_g[w] = r;
        }
        shift = it % m;
        __syncthreads();
      }
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          xp[k] = xr[e];
          gp[k] = gr[e];
        }
      }
      if (tid == 0) st.iter[b] = it + 1;

      // the pairs with rho != 0 (inert pairs have alpha = 0 and leave q
      // unchanged), newest first, listed once so that the recursion's slots
      // and rows are known (and the next row loaded) ahead of each reduction
      if (tid == 0) {
        int nv = 0;
        for (int i = m - 1; i >= 0; --i) {
          int p = i + shift;
          if (p >= m) p -= m;
          const float rho = sh_rho[p];
          if (rho != 0.f) {
            sh_vp[nv] = p;
            sh_vr[nv] = rho;
            ++nv;
          }
        }
        sh_nv = nv;
      }
      __syncthreads();
      const int nv = sh_nv;
      auto row = [&](const float* h, int p, float (&v)[SLOTS]) {
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          v[e] = k < n ? h[(long long)p * n + k] : 0.f;
        }
      };
      // two-loop recursion: q = g; newest to oldest
      float q[SLOTS];
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) q[e] = gr[e];
      float sn[SLOTS];
      if (nv > 0) row(hs, sh_vp[0], sn);
      for (int j = 0; j < nv; ++j) {
        const int p = sh_vp[j];
        float sc[SLOTS], yc[SLOTS];
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) sc[e] = sn[e];
        row(hy, p, yc);
        if (j + 1 < nv) row(hs, sh_vp[j + 1], sn);
        Part<NT, SLOTS> d[1];
        d[0].zero();
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) d[0].fma(e, sc[e], q[e]);
        }
        float dt[1];
        block_sum<NT, SLOTS, 1>(d, dt, red, phase);
        const float al = sh_vr[j] * dt[0];
        if (tid == 0) sh_alpha[j] = al;
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) q[e] = fmaf(-al, yc[e], q[e]);
        }
      }
      // H0 = gamma I from the newest valid pair (rho = 1 / y.s when
      // y.s > 1e-8, else 0: never negative or NaN, so the first listed pair)
      float gamma = 1.f;
      if (nv > 0) {
        float sv[SLOTS], yv[SLOTS];
        row(hs, sh_vp[0], sv);
        row(hy, sh_vp[0], yv);
        Part<NT, SLOTS> d[2];
        d[0].zero();
        d[1].zero();
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) {
            d[0].fma(e, sv[e], yv[e]);
            d[1].fma(e, yv[e], yv[e]);
          }
        }
        float dt[2];
        block_sum<NT, SLOTS, 2>(d, dt, red, phase);
        gamma = dt[0] / dt[1];
      }
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) q[e] *= gamma;
      __syncthreads();  // sh_alpha visible
      // oldest to newest
      float yn[SLOTS];
      if (nv > 0) row(hy, sh_vp[nv - 1], yn);
      for (int j = nv - 1; j >= 0; --j) {
        const int p = sh_vp[j];
        float yc[SLOTS], sc[SLOTS];
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) yc[e] = yn[e];
        row(hs, p, sc);
        if (j > 0) row(hy, sh_vp[j - 1], yn);
        Part<NT, SLOTS> d[1];
        d[0].zero();
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) d[0].fma(e, yc[e], q[e]);
        }
        float dt[1];
        block_sum<NT, SLOTS, 1>(d, dt, red, phase);
        const float coef = sh_alpha[j] - sh_vr[j] * dt[0];
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const int k = tid + NT * e;
          if (k < n) q[e] = fmaf(sc[e], coef, q[e]);
        }
      }
      // direction and the clipped candidates of Alg. 1
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int k = tid + NT * e;
        if (k < n) {
          const float dk = -q[e];
          dir[k] = dk;
          for (int l = 0; l < na; ++l) {
            float v = fmaf(a.prm.alpha[l], dk, xr[e]);
            v = fminf(fmaxf(v, lo[e]), hi[e]);
            cand[(long long)l * n + k] = v;
          }
        }
      }
    }
  }
}

// Seeds of at most N <= 32 variables (IK, very short horizons), one thread
// per seed.  A dot product is formed exactly as the one-warp kernel forms it
// (lane k holds fma(a_k, b_k, 0) for k < n and +0 beyond; lane 0's xor
// butterfly adds lane o's partial to its own for o = 16, 8, 4, 2, 1; the
// virtual-warp sum is 0 + w_0 + 0 + ... + 0), and every element update is
// the same fma, so a seed's result is bit-identical to k_opt<32, 1> and
// hence to every other width.
template <int N>
__device__ __forceinline__ float lane_dot(const float (&a)[N], const float (&b)[N], int n) {
  float p[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) p[k] = k < N && k < n ? fmaf(a[k < N ? k : 0], b[k < N ? k : 0], 0.f) : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int l = 0; l < o; ++l) p[l] = p[l] + p[l + o];
  float s = 0.f;
  s += p[0];
#pragma unroll
  for (int w = 1; w < kVirt / 32; ++w) s += 0.f;
  return s;
}

template <int N>
__device__ __forceinline__ void lane_load(float (&v)[N], const float* src, int n) {
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = k < n ? src[k] : 0.f;
}

template <int N>
__global__ void __launch_bounds__(128) k_opt_lane(const __grid_constant__ OptArgs a) {
  const int D = a.dof, m = a.prm.history, na = a.prm.n_alpha;
  const cr_opt_state& st = a.st;
  pdl_wait();
  pdl_launch_dependents();
  if (a.reset_queue && blockIdx.x == 0 && threadIdx.x == 0) *a.reset_queue = 0;
  for (int bt = blockIdx.x * blockDim.x + threadIdx.x; bt < a.n_seeds; bt += gridDim.x * blockDim.x) {
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
    float xr[N], gr[N];
    lane_load(xr, x, n);
    lane_load(gr, g, n);

    // ---------------- line-search selection (Alg. 1) ----------------
    if (a.do_select) {
      float dr[N];
      lane_load(dr, st.dir + vo, n);
      const float* cand = st.cand + (long long)vo * na;
      const float* cgrad = st.cand_grad + (long long)vo * na;
      const float c0 = st.c[b];
      const float gd0 = lane_dot(gr, dr, n);
      int idx = 0;
      float cnew = st.cand_cost[b * na];
      for (int l = 0; l < na; ++l) {
        const float cl = st.cand_cost[b * na + l];
        bool ok = cl <= c0 + a.prm.armijo_c1 * a.prm.alpha[l] * gd0;
        if (a.prm.flags & CR_WOLFE) {
          float gl[N];
          lane_load(gl, cgrad + (long long)l * n, n);
          const float gld = lane_dot(gl, dr, n);
          if (a.prm.flags & CR_STRONG_WOLFE)
            ok = ok && fabsf(gld) <= a.prm.wolfe_c2 * fabsf(gd0);
          else
            ok = ok && gld >= a.prm.wolfe_c2 * gd0;
        }
        if (ok) {  // largest passing index; 0 when none passes
          idx = l;
          cnew = cl;
        }
      }
      const bool better = cnew < st.best_c[b];  // NaN never improves the best
      lane_load(xr, cand + (long long)idx * n, n);
      lane_load(gr, cgrad + (long long)idx * n, n);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (k < n) {
          x[k] = xr[k];
          g[k] = gr[k];
          if (better) st.best_x[vo + k] = xr[k];
        }
      }
      st.c[b] = cnew;
      st.ls_index[b] = idx;
      if (better) {
        st.best_c[b] = cnew;
        st.best_cfree[b] = st.cand_cfree[b * na + idx];
      }
    }
    if (a.init_best) {
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k < n) st.best_x[vo + k] = xr[k];
      st.best_c[b] = st.c[b];
    }

    // ---------------- L-BFGS step (App. A.7) ----------------
    if (a.do_propose) {
      float* s_g = st.s + (long long)vo * m;
      float* y_g = st.y + (long long)vo * m;
      float* rho_g = st.rho + b * m;
      const int it = st.iter[b];
      int shift = 0;
      if (it > 0) {
        const int w = (it - 1) % m;
        float sv[N], yv[N], xp[N], gp[N];
        lane_load(xp, st.x_prev + vo, n);
        lane_load(gp, st.g_prev + vo, n);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          sv[k] = k < n ? xr[k] - xp[k] : 0.f;
          yv[k] = k < n ? gr[k] - gp[k] : 0.f;
          if (k < n) {
            s_g[(long long)w * n + k] = sv[k];
            y_g[(long long)w * n + k] = yv[k];
          }
        }
        const float ys = lane_dot(yv, sv, n);
        rho_g[w] = ys > 1e-8f ? 1.f / ys : 0.f;
        shift = it % m;
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (k < n) {
          st.x_prev[vo + k] = xr[k];
          st.g_prev[vo + k] = gr[k];
        }
      }
      st.iter[b] = it + 1;

      // two-loop recursion: q = g; newest to oldest
      float q[N];
#pragma unroll
      for (int k = 0; k < N; ++k) q[k] = gr[k];
      float alpha[CR_MAX_HISTORY];
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        const float rho = rho_g[p];
        if (rho == 0.f) {  // inert pair: alpha = 0, q unchanged
          alpha[i] = 0.f;
          continue;
        }
        float sp[N], yp[N];
        lane_load(sp, s_g + (long long)p * n, n);
        lane_load(yp, y_g + (long long)p * n, n);
        const float al = rho * lane_dot(sp, q, n);
        alpha[i] = al;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < n) q[k] = fmaf(-al, yp[k], q[k]);
      }
      // H0 = gamma I from the newest valid pair
      float gamma = 1.f;
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        if (rho_g[p] > 0.f) {
          float sp[N], yp[N];
          lane_load(sp, s_g + (long long)p * n, n);
          lane_load(yp, y_g + (long long)p * n, n);
          gamma = lane_dot(sp, yp, n) / lane_dot(yp, yp, n);
          break;
        }
      }
#pragma unroll
      for (int k = 0; k < N; ++k) q[k] *= gamma;
      for (int i = 0; i < m; ++i) {
        const int p = (i + shift) % m;
        const float rho = rho_g[p];
        if (rho == 0.f) continue;
        float sp[N], yp[N];
        lane_load(sp, s_g + (long long)p * n, n);
        lane_load(yp, y_g + (long long)p * n, n);
        const float coef = alpha[i] - rho * lane_dot(yp, q, n);
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < n) q[k] = fmaf(sp[k], coef, q[k]);
      }
      // direction and the clipped candidates of Alg. 1
      float* dir = st.dir + vo;
      float* cand = st.cand + (long long)vo * na;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (k < n) {
          const float dk = -q[k];
          dir[k] = dk;
          const float lo = a.q_lo[k % D], hi = a.q_hi[k % D];
          for (int l = 0; l < na; ++l) {
            float v = fmaf(a.prm.alpha[l], dk, xr[k]);
            v = fminf(fmaxf(v, lo), hi);
            cand[(long long)l * n + k] = v;
          }
        }
      }
    }
  }
}

// Seeds of at most 8 variables (IK of arms with up to 8 joints), eight lanes
// per seed, lane k holding element k.  The one-warp kernel's sum of 32 lanes
// has +0 in lanes 8..31, so lane 0's butterfly adds +0 twice to each of the
// first eight partials before the levels 4, 2, 1 that combine them; the
// eight-lane group does exactly that, then the same virtual-warp sum, so the
// results are bit-identical to the other widths.
__device__ __forceinline__ float g8_dot(float a, float b, bool live, unsigned gm) {
  float v = live ? fmaf(a, b, 0.f) : 0.f;
  v = (v + 0.f) + 0.f;
  v += __shfl_xor_sync(gm, v, 4, 8);
  v += __shfl_xor_sync(gm, v, 2, 8);
  v += __shfl_xor_sync(gm, v, 1, 8);
  float s = 0.f;
  s += v;
#pragma unroll
  for (int w = 1; w < kVirt / 32; ++w) s += 0.f;
  return s;
}

__global__ void __launch_bounds__(128) k_opt_g8(const __grid_constant__ OptArgs a) {
  const int D = a.dof, m = a.prm.history, na = a.prm.n_alpha;
  const cr_opt_state& st = a.st;
  const int k = threadIdx.x & 7;
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  pdl_wait();
  pdl_launch_dependents();
  if (a.reset_queue && blockIdx.x == 0 && threadIdx.x == 0) *a.reset_queue = 0;
  const int groups = gridDim.x * (blockDim.x >> 3);
  // the eight lanes of a seed take the same trip through this loop
  for (int bt = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; bt < a.n_seeds; bt += groups) {
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
    const bool live = k < n;
    float* x = st.x + vo;
    float* g = st.g + vo;
    float xr = live ? x[k] : 0.f, gr = live ? g[k] : 0.f;

    // ---------------- line-search selection (Alg. 1) ----------------
    if (a.do_select) {
      const float dr = live ? st.dir[vo + k] : 0.f;
      const float* cand = st.cand + (long long)vo * na;
      const float* cgrad = st.cand_grad + (long long)vo * na;
      const float c0 = st.c[b];
      const float gd0 = g8_dot(gr, dr, live, gm);
      int idx = 0;
      float cnew = st.cand_cost[b * na];
      for (int l = 0; l < na; ++l) {
        const float cl = st.cand_cost[b * na + l];
        bool ok = cl <= c0 + a.prm.armijo_c1 * a.prm.alpha[l] * gd0;
        if (a.prm.flags & CR_WOLFE) {
          const float gl = live ? cgrad[(long long)l * n + k] : 0.f;
          const float gld = g8_dot(gl, dr, live, gm);
          if (a.prm.flags & CR_STRONG_WOLFE)
            ok = ok && fabsf(gld) <= a.prm.wolfe_c2 * fabsf(gd0);
          else
            ok = ok && gld >= a.prm.wolfe_c2 * gd0;
        }
        if (ok) {  // largest passing index; 0 when none passes
          idx = l;
          cnew = cl;
        }
      }
      const bool better = cnew < st.best_c[b];  // NaN never improves the best
      if (live) {
        xr = cand[(long long)idx * n + k];
        gr = cgrad[(long long)idx * n + k];
        x[k] = xr;
        g[k] = gr;
        if (better) st.best_x[vo + k] = xr;
      }
      __syncwarp(gm);  // every lane has read best_c before lane 0 writes it
      if (k == 0) {
        st.c[b] = cnew;
        st.ls_index[b] = idx;
        if (better) {
          st.best_c[b] = cnew;
          st.best_cfree[b] = st.cand_cfree[b * na + idx];
        }
      }
    }
    if (a.init_best) {
      if (live) st.best_x[vo + k] = xr;
      __syncwarp(gm);
      if (k == 0) st.best_c[b] = st.c[b];
    }

    // ---------------- L-BFGS step (App. A.7) ----------------
    if (a.do_propose) {
      float* s_g = st.s + (long long)vo * m;
      float* y_g = st.y + (long long)vo * m;
      float* rho_g = st.rho + b * m;
      const int it = st.iter[b];
      int shift = 0;
      __syncwarp(gm);  // every lane has read iter and rho before lane 0 writes them
      if (it > 0) {
        const int w = (it - 1) % m;
        const float xp = live ? st.x_prev[vo + k] : 0.f, gp = live ? st.g_prev[vo + k] : 0.f;
        const float sv = live ? xr - xp : 0.f, yv = live ? gr - gp : 0.f;
        if (live) {
          s_g[(long long)w * n + k] = sv;
          y_g[(long long)w * n + k] = yv;
        }
        const float ys = g8_dot(yv, sv, live, gm);
        if (k == 0) rho_g[w] = ys > 1e-8f ? 1.f / ys : 0.f;
        shift = it % m;
      }
      if (live) {
        st.x_prev[vo + k] = xr;
        st.g_prev[vo + k] = gr;
      }
      __syncwarp(gm);  // the new pair and its rho are visible to the group
      if (k == 0) st.iter[b] = it + 1;

      // two-loop recursion: q = g; newest to oldest
      float q = gr;
      float alpha[CR_MAX_HISTORY];
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        const float rho = rho_g[p];
        if (rho == 0.f) {  // inert pair: alpha = 0, q unchanged
          alpha[i] = 0.f;
          continue;
        }
        const float sp = live ? s_g[(long long)p * n + k] : 0.f, yp = live ? y_g[(long long)p * n + k] : 0.f;
        const float al = rho * g8_dot(sp, q, live, gm);
        alpha[i] = al;
        if (live) q = fmaf(-al, yp, q);
      }
      // H0 = gamma I from the newest valid pair
      float gamma = 1.f;
      for (int i = m - 1; i >= 0; --i) {
        const int p = (i + shift) % m;
        if (rho_g[p] > 0.f) {
          const float sp = live ? s_g[(long long)p * n + k] : 0.f, yp = live ? y_g[(long long)p * n + k] : 0.f;
          gamma = g8_dot(sp, yp, live, gm) / g8_dot(yp, yp, live, gm);
          break;
        }
      }
      q *= gamma;
      for (int i = 0; i < m; ++i) {
        const int p = (i + shift) % m;
        const float rho = rho_g[p];
        if (rho == 0.f) continue;
        const float sp = live ? s_g[(long long)p * n + k] : 0.f, yp = live ? y_g[(long long)p * n + k] : 0.f;
        const float coef = alpha[i] - rho * g8_dot(yp, q, live, gm);
        if (live) q = fmaf(sp, coef, q);
      }
      // direction and the clipped candidates of Alg. 1
      if (live) {
        const float dk = -q;
        st.dir[vo + k] = dk;
        float* cand = st.cand + (long long)vo * na;
        const float lo = a.q_lo[k % D], hi = a.q_hi[k % D];
        for (int l = 0; l < na; ++l) {
          float v = fmaf(a.prm.alpha[l], dk, xr);
          v = fminf(fmaxf(v, lo), hi);
          cand[(long long)l * n + k] = v;
        }
      }
    }
  }
}

// The largest dynamic shared memory any launch may ask for is set once per
// kernel and device (never lowered), so launches captured in a graph stay
// valid whatever is launched later.
template <int NT, int SLOTS>
cudaError_t allow_opt_smem() {
  static unsigned done = 0;  // bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  if (done & bit) return cudaSuccess;
  // 200 KB covers every accepted history * horizon * dof and stays below the
  // opt-in limit together with the kernel's static shared memory
  cudaError_t e =
      cudaFuncSetAttribute(k_opt<NT, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) done |= bit;
  return e;
}

template <int NT, int SLOTS>
cudaError_t launch_opt_as(const OptArgs& a, int smem, cudaStream_t stream) {
  cudaError_t e = allow_opt_smem<NT, SLOTS>();
  if (e != cudaSuccess) return e;
  return launch_pdl(k_opt<NT, SLOTS>, a.n_seeds, NT, (size_t)smem, stream, a);
}

}  // namespace

int opt_smem_bytes(int history, int n_max) { return 2 * history * n_max * (int)sizeof(float); }

cudaError_t launch_opt(const OptArgs& a, int n_max, cudaStream_t stream) {
  if (a.n_seeds <= 0) return cudaSuccess;
  if (n_max > kMaxN) return cudaErrorInvalidValue;
  const int smem = a.do_propose ? opt_smem_bytes(a.prm.history, n_max) : 0;
  // many seeds of at most 32 variables: one thread per seed (throughput);
  // few: one warp per seed (latency); both give the same bits
  if (n_max <= 32 && a.n_seeds >= kLaneSeedsFrom) {
    const int grid = (a.n_seeds + 127) / 128;
    if (n_max <= 8) {
      const long long g8 = ((long long)a.n_seeds * 8 + 127) / 128;
      return launch_pdl(k_opt_g8, (int)(g8 < (1ll << 30) ? g8 : (1ll << 30)), 128, 0, stream, a);
    }
    if (n_max <= 16) return launch_pdl(k_opt_lane<16>, grid, 128, 0, stream, a);
    return launch_pdl(k_opt_lane<32>, grid, 128, 0, stream, a);
  }
  if (n_max <= 32) return launch_opt_as<32, 1>(a, smem, stream);
  if (n_max <= 64) return launch_opt_as<32, 2>(a, smem, stream);
  if (n_max <= 128) return launch_opt_as<32, 4>(a, smem, stream);
  if (n_max <= kVirt) return launch_opt_as<32, 8>(a, smem, stream);
  if (n_max <= 2 * kVirt) return launch_opt_as<kVirt, 2>(a, smem, stream);
  if (n_max <= 4 * kVirt) return launch_opt_as<kVirt, 4>(a, smem, stream);
  return launch_opt_as<kVirt, 8>(a, smem, stream);
}

}  // namespace crgb
