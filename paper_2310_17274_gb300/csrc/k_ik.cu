// k_ik.cu -- cost and gradient of IK-mode evaluations, one thread per
// trajectory, for sm_103a.
//
// In IK mode (the IK problem of Sec. 4 and the single-state checks of the
// steering step of Sec. 5) the states of a trajectory do not interact: no
// sweep, no speed metric, no stencils.  A state's cost is the discrete world
// term (Eq. 10 summed over the boxes, Eq. 11 with speed 1), the self term
// (Eq. 9), the position bound (Eq. 17) and, at the last state, the pose goal
// (Eq. 14) and the joint-space goal (Eq. 15).  With nothing shared between
// the states of a tile, a thread owns a trajectory (usually one state): its
// link transforms sit in its own slice of shared memory, the robot and the
// boxes are read through the read-only data cache (the lanes of a warp
// usually share a problem, so these are broadcasts), and no barrier is needed
// after the robot is staged.  Every sum has one sequential order per thread,
// so a trajectory's result does not depend on the launch.
#include <cuda_runtime.h>
#include <math.h>

#include "crgb_internal.cuh"
#include "k_device.cuh"

namespace crgb {

namespace {

// threads of a CTA: with gradients 96 (five CTAs fit an SM by registers and
// shared memory), cost only 128
constexpr int kIkThreadsGrad = 96;
constexpr int kIkThreadsCost = 128;
constexpr int kNear = 8;         // near spheres of one link kept in registers by the self term
constexpr int kIkSplit = 8;      // threads per trajectory in small launches
constexpr long long kIkSplitBelow = 16384;  // trajectories below which a launch is small

// TPT threads share a trajectory (consecutive lanes): thread `sub` takes the
// links l with l % TPT == sub for the world term and the link pairs g with
// g % TPT == sub for the self term; the partial results are combined in link
// order (costs, gradients) or by an order-free rule (the deepest pair, the
// collision-free flag), so every TPT gives the same bits.  Large launches use
// TPT = 1 (throughput), small ones TPT = 8 (latency).
template <int NT, int TPT, bool GRAD>
__global__ void __launch_bounds__(NT, NT == kIkThreadsGrad ? 5 : 1) k_eval_ik(const __grid_constant__ EvalArgs a) {
  static_assert(TPT == 1 || TPT == 2 || TPT == 4 || TPT == 8 || TPT == 16, "TPT");
  constexpr int kOwn = (kMaxDof + TPT - 1) / TPT;  // links a thread can own
  // rows of this thread's link transforms, s_tf[(l * 3 + row) * NT + tid],
  // then its link bounding-sphere centres, s_lc[l * NT + tid] (w: radius)
  extern __shared__ float4 s_tf[];
  float4* s_lc = s_tf + a.rb.dof * 3 * NT;
  __shared__ float s_fix[(kMaxDof + 1) * 12];
  __shared__ int s_axis[kMaxDof];

  const int D = a.rb.dof, M = a.rb.n_spheres, P = a.rb.n_pairs, G = a.rb.n_groups;
  const int tid = threadIdx.x;
  for (int k = tid; k < (D + 1) * 12; k += NT) s_fix[k] = a.rb.fixed_tf[k];
  for (int k = tid; k < D; k += NT) s_axis[k] = a.rb.axis[k];
  // the robot is constant; theta and the outputs belong to the previous grid
  // until it has finished
  pdl_wait();
  // a small launch (one wave) lets the next kernel start at once; a large one
  // only at its end: waiting CTAs of the next kernel slowed its last wave
  // (an IK solve step 215 -> 133 us)
  if (TPT != 1) pdl_launch_dependents();
  __syncthreads();

  const cr_params& prm = a.prm;
  const uint32_t flags = prm.flags;
  const bool selfc = (flags & CR_SELF) != 0;
  const float eta = prm.eta, inv_eta = 1.f / prm.eta;
  const float e2 = prm.eta_bound, inv_e2 = 1.f / prm.eta_bound;
  // the pair table (robots of up to 64 spheres) lets the self term visit only
  // the pairs of spheres that are near the other link
  const int16_t* pair_at = a.rb.pair_at;
  const int sub = TPT == 1 ? 0 : tid % TPT;
  const unsigned gmask = TPT == 1 ? 0xffffffffu : ((1u << TPT) - 1u) << ((tid & 31) & ~(TPT - 1));

  auto row = [&](int l, int r) -> float4 { return s_tf[(l * 3 + r) * NT + tid]; };
  // world position of a point with link-frame centre c on link l
  auto place = [&](int l, float4 c) -> V3 {
    const float4 r0 = row(l, 0), r1 = row(l, 1), r2 = row(l, 2);
    return v3(fmaf(r0.x, c.x, fmaf(r0.y, c.y, fmaf(r0.z, c.z, r0.w))),
              fmaf(r1.x, c.x, fmaf(r1.y, c.y, fmaf(r1.z, c.z, r1.w))),
              fmaf(r2.x, c.x, fmaf(r2.y, c.y, fmaf(r2.z, c.z, r2.w))));
  };

  const int per_tile = a.problems ? a.max_traj : a.traj_per_tile;
  const int n_tiles = a.problems ? a.n_tiles : (a.prob0.n_traj + a.traj_per_tile - 1) / a.traj_per_tile;
  const long long n_threads = (long long)n_tiles * per_tile * TPT;
  // the TPT threads of a trajectory always take the same trip through this loop
  for (long long gs = (long long)blockIdx.x * NT + tid; gs < n_threads; gs += (long long)gridDim.x * NT) {
    const long long slot = gs / TPT;
    const int tile = (int)(slot / per_tile), r = (int)(slot % per_tile);
    const ProblemView* pv;
    int r0, nt;
    if (a.problems) {
      const int4 td = a.tiles[tile];
      pv = a.problems + td.x;
      r0 = td.y;
      nt = td.z;
    } else {
      pv = &a.prob0;
      r0 = tile * a.traj_per_tile;
      nt = min(a.traj_per_tile, a.prob0.n_traj - r0);
    }
    if (r >= nt) continue;
    const int H = pv->horizon, K = pv->n_boxes;
    const BoxRows* boxes = pv->boxes;
    const long long vb = pv->var_base + (long long)(r0 + r) * H * D;
    float tw = 0.f, ts = 0.f, tb = 0.f, tg = 0.f;
    bool free_ok = true;

    for (int t = 0; t < H; ++t) {
      const float* th = a.theta + vb + (long long)t * D;
      float q[kMaxDof];
#pragma unroll
      for (int j = 0; j < kMaxDof; ++j) q[j] = j < D ? th[j] : 0.f;
      // ---- forward kinematics (Sec. 3.1) into this thread's rows (every
      // thread of the trajectory keeps its own copy)
      {
        float T[12] = {1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f};
#pragma unroll
        for (int l = 0; l < kMaxDof; ++l) {
          if (l >= D) break;
          float sn, cs;
          sincosf(q[l], &sn, &cs);
          float N[12];
          fk_joint(s_fix + 12 * l, s_axis[l], sn, cs, T, N);
#pragma unroll
          for (int k = 0; k < 12; ++k) T[k] = N[k];
          s_tf[(l * 3) * NT + tid] = make_float4(N[0], N[1], N[2], N[3]);
          s_tf[(l * 3 + 1) * NT + tid] = make_float4(N[4], N[5], N[6], N[7]);
          s_tf[(l * 3 + 2) * NT + tid] = make_float4(N[8], N[9], N[10], N[11]);
        }
        for (int l = 0; l < D; ++l) {
          const float4 lb = __ldg(&a.rb.link_bs[l]);
          const V3 c = place(l, lb);
          s_lc[l * NT + tid] = make_float4(c.x, c.y, c.z, lb.w);
        }
      }
      // joint j's share of a force gx on point x of a link at or after j
      // (App. E.1 joint table: revolute joint j moves x by a_j x (x - o_j))
      auto joint_share = [&](int j, V3 x, V3 gx) -> float {
        const float4 r0 = row(j, 0), r1 = row(j, 1), r2 = row(j, 2);
        const int ax = s_axis[j];
        const V3 aj = ax == 0 ? v3(r0.x, r1.x, r2.x) : ax == 1 ? v3(r0.y, r1.y, r2.y) : v3(r0.z, r1.z, r2.z);
        return dot(gx, cross(aj, x - v3(r0.w, r1.w, r2.w)));
      };
      // the state's joint gradient, kept by the thread with sub == 0
      float g[kMaxDof];
#pragma unroll
      for (int j = 0; j < kMaxDof; ++j) g[j] = 0.f;
      float tws = 0.f;  // the state's world cost

      // ---- world term (Eq. 10-11, discrete), link by link: the boxes whose
      // bounding sphere is within reach of the link's bounding sphere (64 at
      // a time), then each sphere of the link against those boxes.  Link l
      // gives a cost c_l and a gradient G_l (joints j <= l), both summed over
      // its spheres in order; the state's sums run over l in order.
      float c_own[kOwn], G_own[kOwn][kMaxDof];
#pragma unroll
      for (int k = 0; k < kOwn; ++k) {
        c_own[k] = 0.f;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) G_own[k][j] = 0.f;
      }
      if (K > 0) {
#pragma unroll
        for (int k = 0; k < kOwn; ++k) {
          const int l = sub + k * TPT;
          if (l >= D) break;
          const float4 lc = s_lc[l * NT + tid];
          if (lc.w < 0.f) continue;  // no enabled sphere
          const float reach = lc.w + eta;
          const int s0 = __ldg(&a.rb.link_start[l]), s1 = __ldg(&a.rb.link_start[l + 1]);
          float cl = 0.f;
          float Gl[kMaxDof];
#pragma unroll
          for (int j = 0; j < kMaxDof; ++j) Gl[j] = 0.f;
          for (int c0 = 0; c0 < K; c0 += 64) {
            const int kc = min(64, K - c0);
            unsigned long long m = 0ull;
            for (int kk = 0; kk < kc; ++kk) {
              const BoxRows* bp = boxes + c0 + kk;
              const float4 bc = __ldg(&bp->c);
              const float dx = lc.x - bc.x, dy = lc.y - bc.y, dz = lc.z - bc.z;
              const float rb = (reach + bc.w) * 1.0001f + 1e-6f;
              // bounding spheres apart: the box test below cannot pass
              if (!(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rb * rb)) continue;
              // the link centre's distance to the box: a sphere of the link
              // within eta of the box puts it within reach
              const float4 b0 = __ldg(&bp->r0), b1 = __ldg(&bp->r1), b2 = __ldg(&bp->r2), h = __ldg(&bp->h);
              const float ux = fmaf(b0.x, lc.x, fmaf(b0.y, lc.y, fmaf(b0.z, lc.z, b0.w)));
              const float uy = fmaf(b1.x, lc.x, fmaf(b1.y, lc.y, fmaf(b1.z, lc.z, b1.w)));
              const float uz = fmaf(b2.x, lc.x, fmaf(b2.y, lc.y, fmaf(b2.z, lc.z, b2.w)));
              const float mx = fmaxf(fabsf(ux) - h.x, 0.f), my = fmaxf(fabsf(uy) - h.y, 0.f),
                          mz = fmaxf(fabsf(uz) - h.z, 0.f);
              if (fmaf(mx, mx, fmaf(my, my, mz * mz)) < reach * reach) m |= 1ull << kk;
            }
            if (!m) continue;
            for (int qq = s0; qq < s1; ++qq) {
              const float4 c = __ldg(&a.rb.link_sph4[qq]);
              if (c.w < 0.f) continue;  // disabled sphere
              const V3 x = place(l, c);
              float S = 0.f;
              V3 gs3 = v3(0.f, 0.f, 0.f);
              unsigned long long mm = m;
              while (mm) {
                const int kk = __ffsll((long long)mm) - 1;
                mm &= mm - 1ull;
                const BoxRows* bp = boxes + c0 + kk;
                const float4 b0 = __ldg(&bp->r0), b1 = __ldg(&bp->r1), b2 = __ldg(&bp->r2), h = __ldg(&bp->h);
                const float ux = fmaf(b0.x, x.x, fmaf(b0.y, x.y, fmaf(b0.z, x.z, b0.w)));
                const float uy = fmaf(b1.x, x.x, fmaf(b1.y, x.y, fmaf(b1.z, x.z, b1.w)));
                const float uz = fmaf(b2.x, x.x, fmaf(b2.y, x.y, fmaf(b2.z, x.z, b2.w)));
                {  // farther than radius + eta outside the box: no term, and clear
                  const float mx = fmaxf(fabsf(ux) - h.x, 0.f), my = fmaxf(fabsf(uy) - h.y, 0.f),
                              mz = fmaxf(fabsf(uz) - h.z, 0.f);
                  const float thr = c.w + eta;
                  if (fmaf(mx, mx, fmaf(my, my, mz * mz)) >= thr * thr) continue;
                }
                V3 gu;
                const float phi = sdf_local(ux, uy, uz, h, gu);
                if (!(phi - c.w > 0.f)) free_ok = false;  // clearance of the waypoint
                const float pen = c.w - phi;
                if (pen > -eta) {
                  float sl;
                  S += smooth_dist(pen, eta, inv_eta, sl);
                  // d pen / d u = -grad phi; box frame -> world frame by R = (R^T)^T
                  const V3 gb = (-sl) * gu;
                  gs3.x += fmaf(b0.x, gb.x, fmaf(b1.x, gb.y, b2.x * gb.z));
                  gs3.y += fmaf(b0.y, gb.x, fmaf(b1.y, gb.y, b2.y * gb.z));
                  gs3.z += fmaf(b0.z, gb.x, fmaf(b1.z, gb.y, b2.z * gb.z));
                }
              }
              if (S != 0.f || gs3.x != 0.f || gs3.y != 0.f || gs3.z != 0.f) {
                cl += prm.w_coll * S;
                if (GRAD) {
                  const V3 gx = prm.w_coll * gs3;
#pragma unroll
                  for (int j = 0; j < kMaxDof; ++j) {
                    if (j > l) break;
                    Gl[j] += joint_share(j, x, gx);
                  }
                }
              }
            }
          }
          if (TPT == 1) {  // links come in order: add at once
            tws += cl;
            if (GRAD) {
#pragma unroll
              for (int j = 0; j < kMaxDof; ++j) g[j] += Gl[j];
            }
          } else {
            c_own[k] = cl;
            if (GRAD) {
#pragma unroll
              for (int j = 0; j < kMaxDof; ++j) G_own[k][j] = Gl[j];
            }
          }
        }
      }
      if (TPT > 1) {
        // link l's sums from thread l % TPT, in link order
#pragma unroll
        for (int l = 0; l < kMaxDof; ++l) {
          if (l >= D) break;
          tws += __shfl_sync(gmask, c_own[l / TPT], l % TPT, TPT);
          if (GRAD) {
#pragma unroll
            for (int j = 0; j < kMaxDof; ++j) {
              if (j > l) break;
              g[j] += __shfl_sync(gmask, G_own[l / TPT][j], l % TPT, TPT);
            }
          }
        }
      }
      tw += tws;

      // ---- self term (Eq. 9): link pairs whose bounding spheres are within
      // 1 mm; with the pair table, only the pairs whose two spheres are each
      // within 1 mm of the other link's bounding sphere (a pair within 1 mm
      // has both), else every listed pair of the link pair.  The deepest
      // penetration wins, the first pair of the caller's list on exact ties;
      // every listed pair counts for the collision-free flag.
      float tss = 0.f;  // the state's self cost
      if (P > 0 && !(flags & CR_NO_SELF_CHECK)) {
        float best = 0.f;
        int arg = -1;
        auto take = [&](float pen, int p) {
          if (pen > best) {
            best = pen;
            arg = p;
          } else if (pen == best && pen > 0.f && __ldg(&a.rb.pair_orig[p]) < __ldg(&a.rb.pair_orig[arg])) {
            arg = p;
          }
        };
        auto test_pair = [&](int p, int i, int j) {
          const float4 ci = __ldg(&a.rb.spheres[i]), cj = __ldg(&a.rb.spheres[j]);
          if (ci.w <= 0.f || cj.w <= 0.f) return;
          const V3 d = place(__ldg(&a.rb.sphere_link[i]), ci) - place(__ldg(&a.rb.sphere_link[j]), cj);
          const float d2 = dot(d, d);
          const float rs = ci.w + cj.w, lp = rs + 1e-3f;
          if (d2 >= lp * lp) return;  // more than 1 mm apart
          const float pen = rs - sqrtf(d2);
          if (!(-pen > 0.f)) free_ok = false;
          take(pen, p);
        };
        for (int gi = sub; gi < G; gi += TPT) {
          const int4 gr = __ldg(&a.rb.groups[gi]);
          const float4 la = s_lc[gr.x * NT + tid], lbb = s_lc[gr.y * NT + tid];
          if (la.w < 0.f || lbb.w < 0.f) continue;
          const float dx = la.x - lbb.x, dy = la.y - lbb.y, dz = la.z - lbb.z;
          const float lim = la.w + lbb.w + 1e-3f;
          if (!(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < lim * lim)) continue;
          bool walk = pair_at == nullptr;
          if (!walk) {
            // spheres of link b within 1 mm of link a's bounding sphere, kept
            // in registers (at most kNear; more: walk the list instead)
            float4 xb[kNear];
            int jb[kNear];
            int nbn = 0;
            {
              const float4 r0 = row(gr.y, 0), r1 = row(gr.y, 1), r2 = row(gr.y, 2);
              const int q1 = __ldg(&a.rb.link_start[gr.y + 1]);
              for (int qq = __ldg(&a.rb.link_start[gr.y]); qq < q1; ++qq) {
                const float4 c = __ldg(&a.rb.link_sph4[qq]);
                if (!(c.w > 0.f)) continue;
                const float x = fmaf(r0.x, c.x, fmaf(r0.y, c.y, fmaf(r0.z, c.z, r0.w)));
                const float y = fmaf(r1.x, c.x, fmaf(r1.y, c.y, fmaf(r1.z, c.z, r1.w)));
                const float z = fmaf(r2.x, c.x, fmaf(r2.y, c.y, fmaf(r2.z, c.z, r2.w)));
                const float ex = x - la.x, ey = y - la.y, ez = z - la.z;
                const float li = c.w + la.w + 1e-3f;
                if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < li * li)) continue;
                const int j = __ldg(&a.rb.link_sph[qq]);
#pragma unroll
                for (int k = 0; k < kNear; ++k)
                  if (k == nbn) {
                    xb[k] = make_float4(x, y, z, c.w);
                    jb[k] = j;
                  }
                ++nbn;
              }
            }
            walk = nbn > kNear;
            if (!walk && nbn > 0) {
              // spheres of link a within 1 mm of link b's bounding sphere,
              // each against the listed ones of b
              const float4 r0 = row(gr.x, 0), r1 = row(gr.x, 1), r2 = row(gr.x, 2);
              const int q1 = __ldg(&a.rb.link_start[gr.x + 1]);
              for (int qq = __ldg(&a.rb.link_start[gr.x]); qq < q1; ++qq) {
                const float4 c = __ldg(&a.rb.link_sph4[qq]);
                if (!(c.w > 0.f)) continue;
                const float x = fmaf(r0.x, c.x, fmaf(r0.y, c.y, fmaf(r0.z, c.z, r0.w)));
                const float y = fmaf(r1.x, c.x, fmaf(r1.y, c.y, fmaf(r1.z, c.z, r1.w)));
                const float z = fmaf(r2.x, c.x, fmaf(r2.y, c.y, fmaf(r2.z, c.z, r2.w)));
                const float ex = x - lbb.x, ey = y - lbb.y, ez = z - lbb.z;
                const float li = c.w + lbb.w + 1e-3f;
                if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < li * li)) continue;
                const int i = __ldg(&a.rb.link_sph[qq]);
#pragma unroll
                for (int k = 0; k < kNear; ++k) {
                  if (k >= nbn) break;
                  const float dx = x - xb[k].x, dy = y - xb[k].y, dz = z - xb[k].z;
                  const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                  const float rs = c.w + xb[k].w, lp = rs + 1e-3f;
                  if (d2 >= lp * lp) continue;  // more than 1 mm apart
                  const int p = __ldg(&pair_at[i * M + jb[k]]);
                  if (p < 0) continue;  // not a listed pair
                  const float pen = rs - sqrtf(d2);
                  if (!(-pen > 0.f)) free_ok = false;
                  take(pen, p);
                }
              }
            }
          }
          if (walk) {
            for (int p = gr.z; p < gr.z + gr.w; ++p) {
              const uint32_t pr = __ldg(&a.rb.pairs[p]);
              test_pair(p, (int)(pr & 0xffffu), (int)(pr >> 16));
            }
          }
        }
        if (TPT > 1) {  // the deepest pair over the trajectory's threads (order-free)
#pragma unroll
          for (int o = TPT / 2; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(gmask, best, o, TPT);
            const int oa = __shfl_xor_sync(gmask, arg, o, TPT);
            if (ob > best || (ob == best && ob > 0.f && oa != arg &&
                              __ldg(&a.rb.pair_orig[oa]) < __ldg(&a.rb.pair_orig[arg]))) {
              best = ob;
              arg = oa;
            }
          }
        }
        if (selfc) {
          tss = prm.w_self * best;
          ts += tss;
          if (GRAD && arg >= 0 && sub == 0) {
            const uint32_t pr = __ldg(&a.rb.pairs[arg]);
            const int pi = (int)(pr & 0xffffu), pj = (int)(pr >> 16);
            const int li = __ldg(&a.rb.sphere_link[pi]), lj = __ldg(&a.rb.sphere_link[pj]);
            const V3 xi = place(li, __ldg(&a.rb.spheres[pi])), xj = place(lj, __ldg(&a.rb.spheres[pj]));
            const V3 d = xi - xj;
            const float n = norm(d);
            if (n > 0.f) {
              const float f = prm.w_self / n;
#pragma unroll
              for (int j = 0; j < kMaxDof; ++j) {
                if (j > li) break;
                g[j] += joint_share(j, xi, (-f) * d);
              }
#pragma unroll
              for (int j = 0; j < kMaxDof; ++j) {
                if (j > lj) break;
                g[j] += joint_share(j, xj, f * d);
              }
            }
          }
        }
      }
      if (TPT > 1) free_ok = __all_sync(gmask, free_ok);
      if (sub != 0) continue;  // the rest of the state: one thread
      if (a.state_terms)
        reinterpret_cast<float2*>(a.state_terms)[vb / D + t] = make_float2(tws, tss);

      // ---- Eq. 14 pose goal and Eq. 15 joint-space goal at the last state
      if (t == H - 1) {
        const float4 t0 = row(D - 1, 0), t1 = row(D - 1, 1), t2 = row(D - 1, 2);
        const float T6[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
        const float* Fe = s_fix + D * 12;
        float E[12];
#pragma unroll
        for (int rr = 0; rr < 3; ++rr) {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            float v = fmaf(T6[4 * rr], Fe[cc], fmaf(T6[4 * rr + 1], Fe[4 + cc], T6[4 * rr + 2] * Fe[8 + cc]));
            E[4 * rr + cc] = cc == 3 ? v + T6[4 * rr + 3] : v;
          }
        }
        const V3 e = v3(E[3] - pv->goal_p[0], E[7] - pv->goal_p[1], E[11] - pv->goal_p[2]);
        const float rn = norm(e);
        float tr = 0.f;
#pragma unroll
        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) tr = fmaf(pv->goal_R[aa * 3 + bb], E[aa * 4 + bb], tr);
        const float dq = (3.f - tr) * 0.25f;
        tg += prm.w_goal_pos * logcoshf(prm.k_goal_pos * rn) + prm.w_goal_rot * logcoshf(prm.k_goal_rot * dq);
        if (GRAD) {
          const float fp = rn > 1e-30f ? prm.w_goal_pos * prm.k_goal_pos * tanhf(prm.k_goal_pos * rn) / rn
                                       : prm.w_goal_pos * prm.k_goal_pos * prm.k_goal_pos;
          const V3 dp = fp * e;
          const float fr = -0.25f * prm.w_goal_rot * prm.k_goal_rot * tanhf(prm.k_goal_rot * dq);
          // d cost / d R = fr R_g; its effect on joint j is a_j . sum_c R_c x dR_c
          V3 w = v3(0.f, 0.f, 0.f);
  #pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            const V3 Rc = v3(E[cc], E[4 + cc], E[8 + cc]);
            const V3 Gc = fr * v3(pv->goal_R[cc], pv->goal_R[3 + cc], pv->goal_R[6 + cc]);
            w = w + cross(Rc, Gc);
          }
          const V3 pe = v3(E[3], E[7], E[11]);
  #pragma unroll
          for (int j = 0; j < kMaxDof; ++j) {
            if (j >= D) break;
            const float4 r0 = row(j, 0), r1 = row(j, 1), r2 = row(j, 2);
            const int ax = s_axis[j];
            const V3 aj = ax == 0 ? v3(r0.x, r1.x, r2.x) : ax == 1 ? v3(r0.y, r1.y, r2.y) : v3(r0.z, r1.z, r2.z);
            g[j] += dot(dp, cross(aj, pe - v3(r0.w, r1.w, r2.w))) + dot(aj, w);
          }
        }
        if ((flags & CR_CSPACE_GOAL) && pv->has_goal_q) {
          float r2 = 0.f;
#pragma unroll
          for (int j = 0; j < kMaxDof; ++j) {
            if (j >= D) break;
            const float d = q[j] - pv->goal_q[j];
            r2 = fmaf(d, d, r2);
          }
          tg += prm.w_cspace * logcoshf(prm.k_cspace * r2);
          if (GRAD) {
            const float cq = 2.f * prm.w_cspace * prm.k_cspace * tanhf(prm.k_cspace * r2);
#pragma unroll
            for (int j = 0; j < kMaxDof; ++j) {
              if (j >= D) break;
              g[j] = fmaf(cq, q[j] - pv->goal_q[j], g[j]);
            }
          }
        }
      }

      // ---- Eq. 17 position bound, and the gradient out
#pragma unroll
      for (int j = 0; j < kMaxDof; ++j) {
        if (j >= D) break;
        float sl;
        tb += prm.w_bound * bound_cost(q[j], __ldg(&a.rb.lim[j]), __ldg(&a.rb.lim[D + j]), e2, inv_e2, sl);
        g[j] = fmaf(prm.w_bound, sl, g[j]);
      }
      if (GRAD) {
        float* go = a.grad + vb + (long long)t * D;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
          if (j >= D) break;
          go[j] = g[j];
        }
      }
    }

    if (sub != 0) continue;
    const int gi = pv->traj_base + r0 + r;
    a.cost[gi] = tw + ts + tb + tg;
    if (a.cfree) a.cfree[gi] = (uint8_t)free_ok;
    if (a.terms) {
      float* tt = a.terms + (long long)gi * CR_N_TERMS;
      tt[0] = tw;
      tt[1] = ts;
      tt[2] = tb;
      tt[3] = 0.f;
      tt[4] = tg;
    }
  }
  if (TPT == 1) pdl_launch_dependents();
}

}  // namespace

static int ik_smem(int dof, int nt) { return dof * 4 * nt * (int)sizeof(float4); }

int eval_ik_smem_bytes(int dof) { return ik_smem(dof, kIkThreadsCost); }

// The dynamic shared memory limit is raised once per device to what the
// largest robot needs, never lowered, so captured launches stay valid.
static cudaError_t allow_ik_smem() {
  static unsigned done = 0;  // bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  if (done & bit) return cudaSuccess;
  const int lg = ik_smem(kMaxDof, kIkThreadsGrad), lc = ik_smem(kMaxDof, kIkThreadsCost);
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_eval_ik<kIkThreadsGrad, 1, true>, at, lg);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eval_ik<kIkThreadsGrad, kIkSplit, true>, at, lg);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eval_ik<kIkThreadsCost, 1, false>, at, lc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eval_ik<kIkThreadsCost, kIkSplit, false>, at, lc);
  if (e == cudaSuccess) done |= bit;
  return e;
}

int eval_ik_blocks_per_sm(int dof) {
  int n = 0;
  if (allow_ik_smem() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_ik<kIkThreadsGrad, 1, true>, kIkThreadsGrad,
                                                    ik_smem(dof, kIkThreadsGrad)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int NT, int TPT, bool GRAD>
static cudaError_t launch_ik(const EvalArgs& a, long long n_slots, cudaStream_t stream) {
  const long long want = (n_slots * TPT + NT - 1) / NT;
  const int grid = (int)(want < (1ll << 30) ? want : (1ll << 30));
  return launch_pdl(k_eval_ik<NT, TPT, GRAD>, grid, NT, (size_t)ik_smem(a.rb.dof, NT), stream, a);
}

cudaError_t launch_eval_ik(const EvalArgs& a, cudaStream_t stream) {
  const int per_tile = a.problems ? a.max_traj : a.traj_per_tile;
  const int n_tiles = a.problems ? a.n_tiles : (a.prob0.n_traj + a.traj_per_tile - 1) / a.traj_per_tile;
  const long long n_slots = (long long)n_tiles * per_tile;
  if (n_slots <= 0) return cudaSuccess;
  cudaError_t e = allow_ik_smem();
  if (e != cudaSuccess) return e;
  // few trajectories: several threads each, for latency (same results);
  // cost-only launches (steering, particles) skip every gradient term
  const bool split = n_slots < kIkSplitBelow;
  if (a.grad)
    return split ? launch_ik<kIkThreadsGrad, kIkSplit, true>(a, n_slots, stream)
                 : launch_ik<kIkThreadsGrad, 1, true>(a, n_slots, stream);
  return split ? launch_ik<kIkThreadsCost, kIkSplit, false>(a, n_slots, stream)
               : launch_ik<kIkThreadsCost, 1, false>(a, n_slots, stream);
}

}  // namespace crgb
