// k_eval.cu -- fused cost-and-gradient evaluation over seeds x timesteps, and
// forward kinematics, for sm_103a.
//
// One CTA owns a tile of whole trajectories of one problem: a single
// trajectory (H = 32..128 states), or several short ones (IK-mode launches
// go to k_ik.cu instead).  Everything a trajectory needs stays on
// chip: the link transforms of every state (forward kinematics, Sec. 3.1),
// the per-(state, sphere) swept world sums and their gradients (Sec. 3.3-3.4,
// Eq. 10-11), the self-collision argmax per state (Eq. 9), the stencil
// derivatives (App. A.5) and the joint gradients.  Only theta is read from
// HBM and only cost / gradient / flags are written back.
//
// Work mapping inside a tile: a warp owns a state, a lane owns spheres
// (i = lane, lane + 32, ...).  Boxes are staged in shared memory in chunks and
// read as warp-wide broadcasts; a cheap squared-distance test skips the
// (sphere, box) pairs whose sweep cannot reach the box.  Every reduction has a
// fixed shape (sequential per lane, then an xor butterfly), so a trajectory's
// result does not depend on the tile size, the CTA size or the other work in
// the launch.
#include <cuda_runtime.h>
#include <math.h>

#include "crgb_internal.cuh"
#include "k_device.cuh"

namespace crgb {

namespace {

// penetration test sample in the box frame: accumulates S and the box-frame
// gradient of S w.r.t. the sample (d pen / d u = -grad phi)
struct SweepAcc {
  float S;
  V3 g;
};

__device__ __forceinline__ float sample_pen(const BoxRows& b, float ux, float uy, float uz, float r,
                                            float eta, float inv_eta, SweepAcc& acc, bool& hit) {
  V3 gu;
  float phi = sdf_local(ux, uy, uz, b.h, gu);
  float pen = r - phi;
  hit = pen > -eta;
  if (hit) {
    float sl;
    acc.S += smooth_dist(pen, eta, inv_eta, sl);
    acc.g = acc.g - sl * gu;
  }
  return phi;
}

// MinBlocks = 1: up to 128 registers a thread, sphere positions may be
// cached in shared memory.  MinBlocks = 2: at most 64 registers and no
// position cache, so that two 512-thread CTAs share an SM.
template <int MinBlocks>
__global__ void __launch_bounds__(512, MinBlocks) k_eval(const __grid_constant__ EvalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ProblemView s_prob;
  __shared__ int s_axis[kMaxDof];
  __shared__ int s_next;
  __shared__ int s_nlist;
  __shared__ int s_nll;
  __shared__ int s_nbw;

  const int D = a.rb.dof, M = a.rb.n_spheres, P = a.rb.n_pairs, G = a.rb.n_groups;
  const int GW = (G + 31) / 32;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const cr_params& prm = a.prm;
  const uint32_t flags = prm.flags;
  const bool ik = (flags & CR_IK_MODE) != 0;
  const bool swept = !ik && (flags & CR_SWEPT);
  const bool speed = !ik && (flags & CR_SPEED);
  const bool selfc = (flags & CR_SELF) != 0;
  const bool store_x = a.store_x != 0;
  const float eta = prm.eta, inv_eta = 1.f / prm.eta;
  const float e2 = prm.eta_bound, inv_e2 = 1.f / prm.eta_bound;

  EvalSmem L;
  L.build(D, M, P, G, a.max_traj, a.max_states, nw, store_x);
  float* s_fix = reinterpret_cast<float*>(smem + L.off_fix);
  float* s_lim = reinterpret_cast<float*>(smem + L.off_lim);
  float4* s_sph = reinterpret_cast<float4*>(smem + L.off_sph);
  int* s_link = reinterpret_cast<int*>(smem + L.off_link);
  float* s_soff = reinterpret_cast<float*>(smem + L.off_soff);
  float4* s_lbs = reinterpret_cast<float4*>(smem + L.off_lbs);
  float* s_ldm = reinterpret_cast<float*>(smem + L.off_ldm);
  int* s_lst = reinterpret_cast<int*>(smem + L.off_lst);
  int* s_lsp = reinterpret_cast<int*>(smem + L.off_lsp);
  uint32_t* s_pairs = reinterpret_cast<uint32_t*>(smem + L.off_pairs);
  int4* s_grp = reinterpret_cast<int4*>(smem + L.off_grp);
  float* s_th = reinterpret_cast<float*>(smem + L.off_th);
  float* s_lt = reinterpret_cast<float*>(smem + L.off_lt);
  float2* s_sc = reinterpret_cast<float2*>(smem + L.off_sc);
  float4* s_x = reinterpret_cast<float4*>(smem + L.off_x);
  float4* s_sg = reinterpret_cast<float4*>(smem + L.off_sg);
  uint32_t* s_nz = reinterpret_cast<uint32_t*>(smem + L.off_nz);
  float* s_lm = reinterpret_cast<float*>(smem + L.off_lm);
  const int MW = (M + 31) / 32;
  float4* s_rho = reinterpret_cast<float4*>(smem + L.off_rho);
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem + L.off_mask);  // 2 words per (state, link)
  float* s_stw = reinterpret_cast<float*>(smem + L.off_stw);
  float* s_sts = reinterpret_cast<float*>(smem + L.off_sts);
  int* s_sta = reinterpret_cast<int*>(smem + L.off_sta);
  uint32_t* s_gmask = reinterpret_cast<uint32_t*>(smem + L.off_gmask);
  float4* s_wsph = reinterpret_cast<float4*>(smem + L.off_wsph);
  // world cost of each (state, sphere) from backward pass 1, in the same
  // region once the self term no longer needs it
  float* s_wc = reinterpret_cast<float*>(smem + L.off_wsph);
  float* s_gth = reinterpret_cast<float*>(smem + L.off_gth);
  // until the backward pass: the (state, sphere) items whose gradient can be
  // non-zero, one bit each, set by the sweep and the self term
  uint32_t* s_bwm = reinterpret_cast<uint32_t*>(smem + L.off_gth);
  BoxRows* s_box = reinterpret_cast<BoxRows*>(smem + L.off_box);
  float4* s_ee = reinterpret_cast<float4*>(smem + L.off_ee);
  float* s_sten = reinterpret_cast<float*>(smem + L.off_sten);
  float* s_pb = reinterpret_cast<float*>(smem + L.off_pb);
  float* s_db = reinterpret_cast<float*>(smem + L.off_db);
  float* s_sm = reinterpret_cast<float*>(smem + L.off_sm);
  float* s_goal = reinterpret_cast<float*>(smem + L.off_goal);
  int* s_free = reinterpret_cast<int*>(smem + L.off_free);
  // the sweep's work list lives in the stencil region, unused until later
  uint32_t* s_list = reinterpret_cast<uint32_t*>(smem + L.off_sten);
  const int list_cap = (L.off_pb - L.off_sten) / 12;
  const int bw_cap = (L.off_pb - L.off_sten) / 4;  // the backward pass's list, same region
  // the (state, link) items with boxes in reach: S * D entries in the bound outputs
  int* s_llist = reinterpret_cast<int*>(smem + L.off_pb);

  // robot model, once per CTA
  for (int k = tid; k < (D + 1) * 12; k += nthr) s_fix[k] = a.rb.fixed_tf[k];
  for (int k = tid; k < 5 * D; k += nthr) s_lim[k] = a.rb.lim[k];
  for (int k = tid; k < M; k += nthr) {
    s_sph[k] = a.rb.spheres[k];
    s_link[k] = a.rb.sphere_link[k];
    s_soff[k] = a.rb.sphere_off[k];
  }
  for (int k = tid; k < D; k += nthr) {
    s_lbs[k] = a.rb.link_bs[k];
    s_ldm[k] = a.rb.link_dmax[k];
  }
  for (int k = tid; k <= D; k += nthr) s_lst[k] = a.rb.link_start[k];
  for (int k = tid; k < M; k += nthr) s_lsp[k] = a.rb.link_sph[k];
  for (int k = tid; k < P; k += nthr) s_pairs[k] = a.rb.pairs[k];
  for (int k = tid; k < G; k += nthr) s_grp[k] = a.rb.groups[k];
  for (int k = tid; k < D; k += nthr) s_axis[k] = a.rb.axis[k];
  // the robot is constant; trajectories, the work counter and the outputs
  // belong to the previous grid until it has finished
  pdl_wait();
  pdl_launch_dependents();

  const int n_tiles = a.problems ? a.n_tiles
                                 : (a.prob0.n_traj + a.traj_per_tile - 1) / a.traj_per_tile;

  // Tiles are taken in order from a device counter (persistent launch over
  // uneven problems) or strided by the grid.
  int tile = blockIdx.x;
  if (a.queue) {
    if (tid == 0) s_next = atomicAdd(a.queue, 1);
    __syncthreads();
    tile = s_next;
  }
  for (; tile < n_tiles;) {
    const ProblemView* pv;
    int r0, nt;
    if (a.problems) {
      int4 td = a.tiles[tile];
      pv = a.problems + td.x;
      r0 = td.y;
      nt = td.z;
    } else {
      pv = &a.prob0;
      r0 = tile * a.traj_per_tile;
      nt = min(a.traj_per_tile, a.prob0.n_traj - r0);
    }
    __syncthreads();  // previous tile fully consumed
    {
      const int* src = reinterpret_cast<const int*>(pv);
      int* dst = reinterpret_cast<int*>(&s_prob);
      for (int k = tid; k < (int)(sizeof(ProblemView) / 4); k += nthr) dst[k] = src[k];
    }
    __syncthreads();
    const int H = s_prob.horizon;
    const int K = s_prob.n_boxes;
    // time step and derivative weights of this problem
    const float dt = s_prob.dt, inv2dt = 0.5f / dt;
    const float w_vel = s_prob.w_vel, w_acc = s_prob.w_acc, w_jerk = s_prob.w_jerk;
    const int S = nt * H;
    const long long vbase = s_prob.var_base + (long long)r0 * H * D;

    for (int k = tid; k < S * D; k += nthr) s_th[k] = a.theta[vbase + k];
    for (int k = tid; k < nt; k += nthr) {
      s_free[k] = 1;
      s_goal[k] = 0.f;
    }
    for (int k = tid; k < S * M; k += nthr) s_sg[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = tid; k < S * GW; k += nthr) s_gmask[k] = 0u;
    if (tid == 0) s_nbw = 0;
    for (int k = tid; k < S * MW; k += nthr) {
      s_nz[k] = 0u;
      s_bwm[k] = 0u;
    }
    __syncthreads();
    // joint sines and cosines of every slot, all threads at once
    for (int k = tid; k < (1 + S) * D; k += nthr) {
      const int s = fdiv(k, a.rb.fd_dof), j = k - s * D;
      float sn, cs;
      sincosf(s == 0 ? s_prob.q_start[j] : s_th[(s - 1) * D + j], &sn, &cs);
      s_sc[k] = make_float2(sn, cs);
    }
    __syncthreads();

    // ---- forward kinematics: slot 0 = start state, slot 1 + sigma = state
    // sigma; three threads per slot, one row of the transforms each
    for (int k = tid; k < 3 * (1 + S); k += nthr) {
      const int s = k / 3;
      fk_chain_row(s_fix, s_axis, D, s_sc + s * D, k - 3 * s, s_lt + s * D * 12);
    }
    __syncthreads();

    // slot of timestep tt (0 = start, clamped to H) of trajectory r
    auto slot = [&](int r, int tt) -> int {
      if (tt <= 0) return 0;
      if (tt > H) tt = H;
      return 1 + r * H + tt - 1;
    };
    auto sphere_at = [&](int sl, int i) -> V3 {
      float4 c = s_sph[i];
      return tf_point(s_lt + (sl * D + s_link[i]) * 12, c.x, c.y, c.z);
    };
    // world position of sphere i at slot sl (stored, or from the transforms)
    auto pos = [&](int sl, int i) -> V3 {
      if (store_x) {
        const float4 v = s_x[sl * M + i];
        return v3(v.x, v.y, v.z);
      }
      return sphere_at(sl, i);
    };
    if (store_x) {
      for (int k = tid; k < (1 + S) * M; k += nthr) {
        const int sl = fdiv(k, a.rb.fd_sph), i = k - sl * M;
        const V3 x = sphere_at(sl, i);
        s_x[k] = make_float4(x.x, x.y, x.z, s_sph[i].w);
      }
    }
    // Link bounding-sphere centre at each state and its reach: a box farther
    // than the reach from the centre can add nothing for any sphere of the
    // link.  Every point of the link at offset d from its centre moves by at
    // most |dc| + |dR|_F d to a neighbouring state, so half of that bounds the
    // sweep length L of each of its spheres, and reach = R_link + max(eta, L).
    for (int k = tid; k < S * D; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_dof), l = k - sg * D;
      const int r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
      const float4 lb = s_lbs[l];
      const float* T1 = s_lt + (slot(r, t) * D + l) * 12;
      const V3 c = tf_point(T1, lb.x, lb.y, lb.z);
      float reach = __int_as_float(0xff800000);  // -inf: no enabled sphere
      float Lm = 0.f;
      if (lb.w >= 0.f) {
        if (swept) {
#pragma unroll
          for (int side = -1; side <= 1; side += 2) {
            const float* T2 = s_lt + (slot(r, t + side) * D + l) * 12;
            const V3 c2 = tf_point(T2, lb.x, lb.y, lb.z);
            float f = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
              for (int w = 0; w < 3; ++w) {
                const float d = T2[4 * q + w] - T1[4 * q + w];
                f = fmaf(d, d, f);
              }
            Lm = fmaxf(Lm, 0.5f * (norm(c2 - c) + sqrtf(f) * s_ldm[l]));
          }
        }
        reach = lb.w + fmaxf(eta, Lm);
      }
      s_rho[k] = make_float4(c.x, c.y, c.z, reach);
      s_lm[k] = fmaxf(eta, Lm);  // bounds (thr - radius) of every sphere of the link
    }
    // Eq. 14 pose cost at the last state of each trajectory, on the last
    // threads of the CTA (idle in the link pass above for short tiles)
    for (int r = nthr - 1 - tid; r >= 0 && r < nt; r += nthr) {
      const float* LTt = s_lt + slot(r, H) * D * 12;
      const float* T6 = LTt + (D - 1) * 12;
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
      const V3 e = v3(E[3] - s_prob.goal_p[0], E[7] - s_prob.goal_p[1], E[11] - s_prob.goal_p[2]);
      const float rn = norm(e);
      float tr = 0.f;
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) tr = fmaf(s_prob.goal_R[aa * 3 + bb], E[aa * 4 + bb], tr);
      const float dq = (3.f - tr) * 0.25f;
      s_goal[r] = prm.w_goal_pos * logcoshf(prm.k_goal_pos * rn) +
                  prm.w_goal_rot * logcoshf(prm.k_goal_rot * dq);
      const float fp = rn > 1e-30f ? prm.w_goal_pos * prm.k_goal_pos * tanhf(prm.k_goal_pos * rn) / rn
                                   : prm.w_goal_pos * prm.k_goal_pos * prm.k_goal_pos;
      const V3 dp = fp * e;
      const float fr = -0.25f * prm.w_goal_rot * prm.k_goal_rot * tanhf(prm.k_goal_rot * dq);
      // d cost / d R = fr R_g; its effect on joint j is a_j . sum_c R_c x dR_c
      V3 w = v3(0.f, 0.f, 0.f);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const V3 Rc = v3(E[cc], E[4 + cc], E[8 + cc]);
        const V3 Gc = fr * v3(s_prob.goal_R[cc], s_prob.goal_R[3 + cc], s_prob.goal_R[6 + cc]);
        w = w + cross(Rc, Gc);
      }
      // Eq. 15 joint-space goal term: alpha_4 logcosh(alpha_5 |theta_g - theta_H|^2);
      // its gradient on theta_H is cq (theta_H - theta_g), cq kept beside the pose
      float cq = 0.f;
      if ((flags & CR_CSPACE_GOAL) && s_prob.has_goal_q) {
        const float* thH = s_th + (r * H + H - 1) * D;
        float r2 = 0.f;
        for (int j = 0; j < D; ++j) {
          const float d = thH[j] - s_prob.goal_q[j];
          r2 = fmaf(d, d, r2);
        }
        s_goal[r] += prm.w_cspace * logcoshf(prm.k_cspace * r2);
        cq = 2.f * prm.w_cspace * prm.k_cspace * tanhf(prm.k_cspace * r2);
      }
      s_ee[3 * r] = make_float4(dp.x, dp.y, dp.z, 0.f);
      s_ee[3 * r + 1] = make_float4(w.x, w.y, w.z, 0.f);
      s_ee[3 * r + 2] = make_float4(E[3], E[7], E[11], cq);
    }
    __syncthreads();

    // Neighbour positions of sphere i at state (r, t) for the sweep: half
    // distances L0, L2 to the previous / next waypoint and unit directions.
    // thr = r + max(eta, L0, L2): a box farther than thr from the centre can
    // add nothing (waypoint outside eta, no sweep sample reaches it).
    struct SphereMotion {
      V3 x1, dir0, dir2;
      float L0, L2, thr;
    };
    auto motion = [&](int r, int t, int i) -> SphereMotion {
      SphereMotion mo;
      mo.x1 = pos(slot(r, t), i);
      mo.dir0 = v3(0.f, 0.f, 0.f);
      mo.dir2 = mo.dir0;
      mo.L0 = 0.f;
      mo.L2 = 0.f;
      if (swept) {
        const V3 d0 = pos(slot(r, t - 1), i) - mo.x1;
        const V3 d2 = pos(slot(r, t + 1), i) - mo.x1;
        const float n0 = norm(d0), n2 = norm(d2);
        mo.L0 = 0.5f * n0;
        mo.L2 = 0.5f * n2;
        if (n0 > 0.f) mo.dir0 = (1.f / n0) * d0;
        if (n2 > 0.f) mo.dir2 = (1.f / n2) * d2;
      }
      mo.thr = s_sph[i].w + fmaxf(eta, fmaxf(mo.L0, mo.L2));
      return mo;
    };

    // Self-collision link pairs whose bounding spheres are within 1 mm (the
    // pair search below skips the others); the world term's first barrier
    // publishes the mask.
    for (int k = tid; k < S * G; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_grp), g = k - sg * G;
      const int4 gr = s_grp[g];
      const float4 A = s_rho[sg * D + gr.x], B = s_rho[sg * D + gr.y];
      const float ra = s_lbs[gr.x].w, rb = s_lbs[gr.y].w;
      if (ra >= 0.f && rb >= 0.f) {
        const float dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
        const float lim = ra + rb + 1e-3f;
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < lim * lim) atomicOr(&s_gmask[sg * GW + g / 32], 1u << (g % 32));
      }
    }
    if (K == 0) __syncthreads();

    // ---- world term (Eq. 11 with the sweep of Sec. 3.4)
    if (K > 0) {
      for (int c0 = 0; c0 < K; c0 += kBoxChunk) {
        const int kc = min(kBoxChunk, K - c0);
        __syncthreads();
        {
          const float4* src = reinterpret_cast<const float4*>(s_prob.boxes + c0);
          float4* dst = reinterpret_cast<float4*>(s_box);
          constexpr int kRow = (int)(sizeof(BoxRows) / 16);
          for (int k = tid; k < kc * kRow; k += nthr) dst[k] = src[k];
          if (tid == 0) {
            s_nlist = 0;
            s_nll = 0;
          }
        }
        __syncthreads();
        // (1) per (state, link): bitmask of the boxes within reach
        for (int k = tid; k < S * D; k += nthr) {
          const float4 lc = s_rho[k];
          unsigned long long m = 0ull;
          if (lc.w >= 0.f) {
            const float rr = lc.w * lc.w;
#pragma unroll 4
            for (int kk = 0; kk < kc; ++kk) {
              const BoxRows& b = s_box[kk];
              // bounding spheres apart: the box test below cannot pass
              const float cx = lc.x - b.c.x, cy = lc.y - b.c.y, cz = lc.z - b.c.z;
              const float rb = (lc.w + b.c.w) * 1.0001f + 1e-6f;
              if (fmaf(cx, cx, fmaf(cy, cy, cz * cz)) >= rb * rb) continue;
              const float ux = fmaf(b.r0.x, lc.x, fmaf(b.r0.y, lc.y, fmaf(b.r0.z, lc.z, b.r0.w)));
              const float uy = fmaf(b.r1.x, lc.x, fmaf(b.r1.y, lc.y, fmaf(b.r1.z, lc.z, b.r1.w)));
              const float uz = fmaf(b.r2.x, lc.x, fmaf(b.r2.y, lc.y, fmaf(b.r2.z, lc.z, b.r2.w)));
              const float mx = fmaxf(fabsf(ux) - b.h.x, 0.f);
              const float my = fmaxf(fabsf(uy) - b.h.y, 0.f);
              const float mz = fmaxf(fabsf(uz) - b.h.z, 0.f);
              if (fmaf(mx, mx, fmaf(my, my, mz * mz)) < rr) m |= 1ull << kk;
            }
          }
          s_mask[2 * k] = (uint32_t)m;
          s_mask[2 * k + 1] = (uint32_t)(m >> 32);
          if (m) s_llist[atomicAdd(&s_nll, 1)] = k;  // at most S * D entries: always fits
        }
        __syncthreads();
        // (2) the sweep of a (state, sphere) over the boxes in mask m, in box order
        auto sweep_item = [&](int k, unsigned long long m) {
          const int sg = fdiv(k, a.rb.fd_sph), i = k - sg * M;
          const int r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
          const float rad = s_sph[i].w;
          const SphereMotion mo = motion(r, t, i);
          const V3 x1 = mo.x1;
          float4 acc4 = s_sg[k];
          bool clear = true;
          while (m) {
            const int kk = __ffsll((long long)m) - 1;
            m &= m - 1ull;
            const BoxRows& b = s_box[kk];
            const float ux = fmaf(b.r0.x, x1.x, fmaf(b.r0.y, x1.y, fmaf(b.r0.z, x1.z, b.r0.w)));
            const float uy = fmaf(b.r1.x, x1.x, fmaf(b.r1.y, x1.y, fmaf(b.r1.z, x1.z, b.r1.w)));
            const float uz = fmaf(b.r2.x, x1.x, fmaf(b.r2.y, x1.y, fmaf(b.r2.z, x1.z, b.r2.w)));
            const float mx = fmaxf(fabsf(ux) - b.h.x, 0.f);
            const float my = fmaxf(fabsf(uy) - b.h.y, 0.f);
            const float mz = fmaxf(fabsf(uz) - b.h.z, 0.f);
            if (fmaf(mx, mx, fmaf(my, my, mz * mz)) >= mo.thr * mo.thr) continue;
            // waypoint, then the two half-way sweeps
            SweepAcc sw{0.f, v3(0.f, 0.f, 0.f)};
            bool hit;
            const float phi1 = sample_pen(b, ux, uy, uz, rad, eta, inv_eta, sw, hit);
            if (!(phi1 - rad > 0.f)) clear = false;
            const float u0 = hit ? rad + eta : phi1 - rad;
            if (swept) {
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const float Ls = side == 0 ? mo.L0 : mo.L2;
                if (!(Ls > 0.f)) continue;
                const V3 dw = side == 0 ? mo.dir0 : mo.dir2;
                // direction in the box frame (rotation only)
                const float dx = fmaf(b.r0.x, dw.x, fmaf(b.r0.y, dw.y, b.r0.z * dw.z));
                const float dy = fmaf(b.r1.x, dw.x, fmaf(b.r1.y, dw.y, b.r1.z * dw.z));
                const float dz = fmaf(b.r2.x, dw.x, fmaf(b.r2.y, dw.y, b.r2.z * dw.z));
                float u = u0;
                for (int st = 0; st < prm.sweep_steps; ++st) {
                  if (u >= Ls) break;
                  const float phi = sample_pen(b, fmaf(u, dx, ux), fmaf(u, dy, uy), fmaf(u, dz, uz),
                                               rad, eta, inv_eta, sw, hit);
                  u += hit ? rad + eta : phi - rad;
                }
              }
            }
            // box frame -> world frame: grad_x = R grad_u, R = (R^T)^T
            acc4.x += sw.S;
            acc4.y += fmaf(b.r0.x, sw.g.x, fmaf(b.r1.x, sw.g.y, b.r2.x * sw.g.z));
            acc4.z += fmaf(b.r0.y, sw.g.x, fmaf(b.r1.y, sw.g.y, b.r2.y * sw.g.z));
            acc4.w += fmaf(b.r0.z, sw.g.x, fmaf(b.r1.z, sw.g.y, b.r2.z * sw.g.z));
          }
          s_sg[k] = acc4;
          if (!clear) s_free[r] = 0;
          // the item's gradient, and through the speed its neighbours', can be
          // non-zero (S only grows over box chunks, so the marks cover the end state)
          const uint32_t bit = 1u << (i & 31);
          const int wi = i >> 5;
          if (acc4.x != 0.f || acc4.y != 0.f || acc4.z != 0.f || acc4.w != 0.f) atomicOr(&s_bwm[sg * MW + wi], bit);
          if (speed && acc4.x != 0.f) {
            if (t >= 2) atomicOr(&s_bwm[(sg - 1) * MW + wi], bit);
            if (t + 1 <= H) atomicOr(&s_bwm[(sg + 1) * MW + wi], bit);
          }
        };
        // (2a) per sphere of a listed (state, link): the boxes of the link's mask
        //      within the link-level bound of the sphere; the few items with any
        //      go to a list (inline when the list is full) so that (2b) runs
        //      them densely
        const int n_ll = s_nll, spl = a.rb.max_link_spheres;
        for (int w = tid; w < n_ll * spl; w += nthr) {
          const int wl = fdiv(w, a.rb.fd_lsph);
          const int sl0 = s_llist[wl], jl = w - wl * spl;
          const int sg = fdiv(sl0, a.rb.fd_dof), l = sl0 - sg * D;
          if (jl >= s_lst[l + 1] - s_lst[l]) continue;
          const int i = s_lsp[s_lst[l] + jl];
          const int k = sg * M + i;
          const float4 ci = s_sph[i];
          const float rad = ci.w;
          if (rad < 0.f) continue;
          unsigned long long m0 = (unsigned long long)s_mask[2 * sl0] | ((unsigned long long)s_mask[2 * sl0 + 1] << 32);
          const int r = fdiv(sg, s_prob.fd_h);
          const int sl = slot(r, sg - r * H + 1);
          // sphere i is on link l: its position from link l's transform
          const V3 xp = store_x ? pos(sl, i) : tf_point(s_lt + (sl * D + l) * 12, ci.x, ci.y, ci.z);
          const float tu = rad + s_lm[sl0];
          // boxes within the link-level bound of this sphere's reach, two per
          // step (independent loads; the second one repeats the first when
          // there is none)
          auto near_box = [&](int kk) -> bool {
            const BoxRows& b = s_box[kk];
            const float ux = fmaf(b.r0.x, xp.x, fmaf(b.r0.y, xp.y, fmaf(b.r0.z, xp.z, b.r0.w)));
            const float uy = fmaf(b.r1.x, xp.x, fmaf(b.r1.y, xp.y, fmaf(b.r1.z, xp.z, b.r1.w)));
            const float uz = fmaf(b.r2.x, xp.x, fmaf(b.r2.y, xp.y, fmaf(b.r2.z, xp.z, b.r2.w)));
            const float mx = fmaxf(fabsf(ux) - b.h.x, 0.f);
            const float my = fmaxf(fabsf(uy) - b.h.y, 0.f);
            const float mz = fmaxf(fabsf(uz) - b.h.z, 0.f);
            return fmaf(mx, mx, fmaf(my, my, mz * mz)) < tu * tu;
          };
          unsigned long long m = 0ull;
          while (m0) {
            const int k1 = __ffsll((long long)m0) - 1;
            m0 &= m0 - 1ull;
            const int k2 = m0 ? __ffsll((long long)m0) - 1 : k1;
            m0 &= m0 - 1ull;  // no-op when m0 is 0
            const bool n1 = near_box(k1), n2 = near_box(k2);
            if (n1) m |= 1ull << k1;
            if (n2) m |= 1ull << k2;
          }
          if (!m) continue;
          const int e = atomicAdd(&s_nlist, 1);
          if (e < list_cap) {
            s_list[3 * e] = (uint32_t)k;
            s_list[3 * e + 1] = (uint32_t)m;
            s_list[3 * e + 2] = (uint32_t)(m >> 32);
          } else {
            sweep_item(k, m);
          }
        }
        __syncthreads();
        // (2b) the listed items, any thread: each item keeps its own box order
        {
          const int n_list = min(s_nlist, list_cap);
          for (int e = tid; e < n_list; e += nthr)
            sweep_item((int)s_list[3 * e],
                       (unsigned long long)s_list[3 * e + 1] | ((unsigned long long)s_list[3 * e + 2] << 32));
        }
      }
    }

    // ---- self-collision (Eq. 9): link pairs whose bounding spheres are more
    // than 1 mm apart were skipped above; the rest are searched pair by pair,
    // a warp per state
    for (int sg = warp; sg < S; sg += nw) {
      const int r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
      const int sl = slot(r, t);
      const float4* X = store_x ? s_x + sl * M : s_wsph + warp * M;
      if (!store_x) {
        for (int i = lane; i < M; i += 32) {
          const V3 x = sphere_at(sl, i);
          s_wsph[warp * M + i] = make_float4(x.x, x.y, x.z, s_sph[i].w);
        }
        __syncwarp();
      }
      // deepest penetration and its pair; the caller's pair index (ties: the
      // first pair in the caller's list) is fetched only for exact ties.  A
      // lane takes up to three pairs of a group at once (independent loads).
      float best = 0.f;
      int arg = -1;
      bool touch = false;
      for (int w = 0; w < GW; ++w) {
        uint32_t gm = s_gmask[sg * GW + w];
        while (gm) {
          const int g = w * 32 + __ffs(gm) - 1;
          gm &= gm - 1u;
          const int4 gr = s_grp[g];
          const int end = gr.z + gr.w;
          for (int p0 = gr.z + lane; p0 < end; p0 += 96) {
            uint32_t pr[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) pr[u] = p0 + 32 * u < end ? s_pairs[p0 + 32 * u] : 0u;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const int p = p0 + 32 * u;
              const float4 A = X[pr[u] & 0xffffu], B = X[pr[u] >> 16];
              const float dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
              const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              const float rs = A.w + B.w;
              const float lim = rs + 1e-3f;
              // past the group, disabled spheres, or separated by more than
              // 1 mm: no effect
              if (p >= end || A.w <= 0.f || B.w <= 0.f || d2 >= lim * lim) continue;
              const float pen = rs - sqrtf(d2);
              if (!(-pen > 0.f)) touch = true;
              if (pen > best) {
                best = pen;
                arg = p;
              } else if (pen == best && pen > 0.f && a.rb.pair_orig[p] < a.rb.pair_orig[arg]) {
                arg = p;  // exact tie: first in the caller's list
              }
            }
          }
        }
      }
      // across lanes: the largest penetration (best >= 0, so its bits order
      // as integers), ties to the first pair in the caller's list
      const float bmax = __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(best)));
      int barg = -1;
      if (bmax > 0.f) {
        const bool cand = best == bmax;
        const uint32_t cm = __ballot_sync(0xffffffffu, cand);
        if (__popc(cm) == 1) {
          barg = __shfl_sync(0xffffffffu, arg, __ffs(cm) - 1);
        } else {
          const int ori = cand ? a.rb.pair_orig[arg] : 0x7fffffff;
          const int omin = __reduce_min_sync(0xffffffffu, ori);
          barg = __shfl_sync(0xffffffffu, arg, __ffs(__ballot_sync(0xffffffffu, cand && ori == omin)) - 1);
        }
      }
      touch = __any_sync(0xffffffffu, touch);
      if (lane == 0) {
        s_sts[sg] = bmax;
        s_sta[sg] = barg;
        if (touch) s_free[r] = 0;
        if (selfc && barg >= 0) {  // the deepest pair's spheres carry the self gradient
          const uint32_t pr = s_pairs[barg];
          const int pi = (int)(pr & 0xffffu), pj = (int)(pr >> 16);
          atomicOr(&s_bwm[sg * MW + (pi >> 5)], 1u << (pi & 31));
          atomicOr(&s_bwm[sg * MW + (pj >> 5)], 1u << (pj & 31));
        }
      }
      __syncwarp();
    }
    __syncthreads();

    // ---- backward (App. E.1 Table "Gradient for different joint types":
    // revolute joint j moves a point x by a_j x (x - o_j) and rotates a frame
    // R by [a_j]_x R).
    // (1) per (state, sphere): d cost / d centre from the world term (own
    //     sweep gradient scaled by the speed, plus the speed's dependence on
    //     the neighbouring waypoints) and the self term; it replaces the sweep
    //     gradient in place (the sum S stays for the neighbours)
    auto bw1_item = [&](int k) {
      const int sg = fdiv(k, a.rb.fd_sph), i = k - sg * M;
      const int r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
      const float4 c = s_sph[i];
      float wc = 0.f;
      V3 gx = v3(0.f, 0.f, 0.f);
      if (c.w >= 0.f) {
        const V3 x = pos(slot(r, t), i);
        if (K > 0) {
          const float4 sgv = s_sg[k];
          float v = 1.f;
          if (speed) {
            const V3 d = pos(slot(r, t + 1), i) - pos(slot(r, t - 1), i);
            const float n = norm(d);
            v = n * inv2dt;
            // x_{H+1} := x_H, so the last state's own speed depends on it
            if (t == H && n > 0.f && sgv.x != 0.f) gx = gx + (prm.w_coll * sgv.x * inv2dt / n) * d;
            if (t >= 2) {
              const float Sm = s_sg[k - M].x;
              if (Sm != 0.f) {
                const V3 dm = x - pos(slot(r, t - 2), i);
                const float nm = norm(dm);
                if (nm > 0.f) gx = gx + (prm.w_coll * Sm * inv2dt / nm) * dm;
              }
            }
            if (t + 1 <= H) {
              const float Sp = s_sg[k + M].x;
              if (Sp != 0.f) {
                const V3 dp = pos(slot(r, t + 2), i) - x;
                const float np = norm(dp);
                if (np > 0.f) gx = gx - (prm.w_coll * Sp * inv2dt / np) * dp;
              }
            }
          }
          gx = gx + (prm.w_coll * v) * v3(sgv.y, sgv.z, sgv.w);
          wc = prm.w_coll * v * sgv.x;
        }
        const int parg = selfc ? s_sta[sg] : -1;
        if (parg >= 0) {
          const uint32_t pr = s_pairs[parg];
          const int pi = (int)(pr & 0xffffu), pj = (int)(pr >> 16);
          if (i == pi || i == pj) {
            const V3 d = pos(slot(r, t), pi) - pos(slot(r, t), pj);
            const float n = norm(d);
            if (n > 0.f) {
              const float f = prm.w_self / n;
              gx = gx + (i == pi ? -f : f) * d;
            }
          }
        }
      }
      float* g3 = reinterpret_cast<float*>(&s_sg[k]);
      g3[1] = gx.x;
      g3[2] = gx.y;
      g3[3] = gx.z;
      s_wc[k] = wc;
      if (wc != 0.f || gx.x != 0.f || gx.y != 0.f || gx.z != 0.f)
        atomicOr(&s_nz[sg * MW + i / 32], 1u << (i % 32));
    };
    // (1a) list the (state, sphere) items whose gradient can be non-zero
    //      (marked by the sweep and the self term: own sweep result, a
    //      neighbour's sweep sum through the speed, the deepest self pair);
    //      nothing reaches the others, their gradient and cost stay zero
    // (a strided scan, so that the items past the list's capacity, run by
    //  the thread that finds them, are spread over the CTA)
    for (int k = tid; k < S * M; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_sph), i = k - sg * M;
      if (!((s_bwm[sg * MW + (i >> 5)] >> (i & 31)) & 1u)) continue;
      const int e = atomicAdd(&s_nbw, 1);
      if (e < bw_cap)
        s_list[e] = (uint32_t)k;
      else
        bw1_item(k);
    }
    __syncthreads();
    // (1b) the listed items, any thread
    {
      const int n_list = min(s_nbw, bw_cap);
      for (int e = tid; e < n_list; e += nthr) bw1_item((int)s_list[e]);
    }
    __syncthreads();
    // (2) Jacobian transpose in suffix form: joint j's sum over the spheres on
    //     links at or after j of gx . (a_j x (x - o_j)) equals
    //     a_j . (sum_{l >= j} P_l - o_j x sum_{l >= j} F_l) with, per link l,
    //     P_l = sum x x gx and F_l = sum gx over its non-zero spheres.
    // (2a) per (state, link): P_l and F_l in sphere order, in the region of the
    //      link centres and box masks (unused since the collision terms)
    float* s_pf = reinterpret_cast<float*>(smem + L.off_rho);  // [S][dof][6]
    for (int k = tid; k < S * D; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_dof), l = k - sg * D;
      const int rr = fdiv(sg, s_prob.fd_h);
      const int sl = slot(rr, sg - rr * H + 1);
      V3 P = v3(0.f, 0.f, 0.f), F = v3(0.f, 0.f, 0.f);
      for (int q = s_lst[l]; q < s_lst[l + 1]; ++q) {
        const int i = s_lsp[q];
        if (!((s_nz[sg * MW + (i >> 5)] >> (i & 31)) & 1u)) continue;
        const float4 g = s_sg[sg * M + i];
        const V3 gv = v3(g.y, g.z, g.w);
        P = P + cross(pos(sl, i), gv);
        F = F + gv;
      }
      float* o = s_pf + 6 * k;
      o[0] = P.x; o[1] = P.y; o[2] = P.z;
      o[3] = F.x; o[4] = F.y; o[5] = F.z;
    }

    // ---- Eq. 17 position bound; App. A.5 stencils with Eq. 16 and Eq. 17 on v, a, j
    const int NS = H + 1;
    for (int k = tid; k < S * D; k += nthr) {
      const int j = k - fdiv(k, a.rb.fd_dof) * D;
      float sl;
      s_pb[k] = prm.w_bound * bound_cost(s_th[k], s_lim[j], s_lim[D + j], e2, inv_e2, sl);
    }
    // padded sequence of App. A.2: 3 copies of q_start, theta_1..theta_H, 2 copies of theta_H
    auto ext = [&](int r, int n, int j) -> float {
      if (n <= 2) return s_prob.q_start[j];
      if (n >= H + 2) return s_th[(r * H + H - 1) * D + j];
      return s_th[(r * H + n - 3) * D + j];
    };
    const float inv12dt = 1.f / (12.f * dt), inv12dt2 = 1.f / (12.f * dt * dt),
                inv2dt3 = 1.f / (2.f * dt * dt * dt);
    if (!ik) {
      for (int k = tid; k < nt * NS * D; k += nthr) {
        const int r = fdiv(k, s_prob.fd_hd), rem = k - r * (NS * D), e0 = fdiv(rem, a.rb.fd_dof), e = e0 + 2, j = rem - e0 * D;
        const float qm2 = ext(r, e - 2, j), qm1 = ext(r, e - 1, j), q0 = ext(r, e, j),
                    qp1 = ext(r, e + 1, j), qp2 = ext(r, e + 2, j);
        const float vel = (qm2 - 8.f * qm1 + 8.f * qp1 - qp2) * inv12dt;
        const float accl = (-qm2 + 16.f * qm1 - 30.f * q0 + 16.f * qp1 - qp2) * inv12dt2;
        const float jrk = (-qm2 + 2.f * qm1 - 2.f * qp1 + qp2) * inv2dt3;
        float sm = w_acc * accl * accl + w_jerk * jrk * jrk;
        float dv = 0.f, da = 2.f * w_acc * accl, dj = 2.f * w_jerk * jrk;
        if (flags & CR_VEL_COST) {
          sm += w_vel * logcoshf(prm.k_vel * vel);
          dv += w_vel * prm.k_vel * tanhf(prm.k_vel * vel);
        }
        float s1, s2, s3;
        const float vm = s_lim[2 * D + j], am = s_lim[3 * D + j], jm = s_lim[4 * D + j];
        const float db = bound_cost(vel, -vm, vm, e2, inv_e2, s1) +
                         bound_cost(accl, -am, am, e2, inv_e2, s2) +
                         bound_cost(jrk, -jm, jm, e2, inv_e2, s3);
        dv += prm.w_bound * s1;
        da += prm.w_bound * s2;
        dj += prm.w_bound * s3;
        s_sten[3 * k] = dv;
        s_sten[3 * k + 1] = da;
        s_sten[3 * k + 2] = dj;
        s_sm[k] = sm;
        s_db[k] = prm.w_bound * db;
      }
    }
    __syncthreads();
    // (2b) per (state, joint): the suffix sums and the end-effector terms;
    //      per state, on the last threads of the CTA (idle here when S D is
    //      below the CTA size), the state's world cost in sphere order
    for (int k = tid; k < S * D; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_dof), j = k - sg * D;
      const int r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
      const int sl = slot(r, t);
      const float* T = s_lt + (sl * D + j) * 12;
      const int ax = s_axis[j];
      const V3 aj = v3(T[ax], T[4 + ax], T[8 + ax]);
      const V3 oj = v3(T[3], T[7], T[11]);
      V3 Ps = v3(0.f, 0.f, 0.f), Fs = v3(0.f, 0.f, 0.f);
      for (int l = j; l < D; ++l) {
        const float* p = s_pf + 6 * (sg * D + l);
        Ps = Ps + v3(p[0], p[1], p[2]);
        Fs = Fs + v3(p[3], p[4], p[5]);
      }
      float acc = dot(aj, Ps) - dot(aj, cross(oj, Fs));
      if (t == H) {
        const float4 dp = s_ee[3 * r], w = s_ee[3 * r + 1], pe = s_ee[3 * r + 2];
        acc += dot(v3(dp.x, dp.y, dp.z), cross(aj, v3(pe.x, pe.y, pe.z) - oj)) + dot(aj, v3(w.x, w.y, w.z));
      }
      s_gth[k] = acc;
    }
    for (int sg = nthr - 1 - tid; sg >= 0 && sg < S; sg += nthr) {
      float wsum = 0.f;
      if (K > 0) {
        for (int w = 0; w < MW; ++w) {
          uint32_t bits = s_nz[sg * MW + w];
          while (bits) {
            const int i = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            // world cost of the sphere (beta_2 speed S, from backward pass 1)
            if (s_sg[sg * M + i].x != 0.f) wsum += s_wc[sg * M + i];
          }
        }
      }
      s_stw[sg] = wsum;
    }
    __syncthreads();

    // ---- gradient: kinematic part + position bound + stencil transpose
    for (int k = tid; k < S * D; k += nthr) {
      const int sg = fdiv(k, a.rb.fd_dof), j = k - sg * D, r = fdiv(sg, s_prob.fd_h), t = sg - r * H + 1;
      float sl;
      bound_cost(s_th[k], s_lim[j], s_lim[D + j], e2, inv_e2, sl);
      float g = s_gth[k] + prm.w_bound * sl;
      if (t == H) g = fmaf(s_ee[3 * r + 2].w, s_th[k] - s_prob.goal_q[j], g);  // Eq. 15
      if (!ik) {
        const int nhi = t == H ? H + 4 : t + 2;
        for (int n = t + 2; n <= nhi; ++n) {
          const int elo = max(2, n - 2), ehi = min(H + 2, n + 2);
          for (int e = elo; e <= ehi; ++e) {
            const int o = n - e;  // position of theta in the stencil of sample e
            const float* sd = s_sten + 3 * ((r * NS + e - 2) * D + j);
            const float cv = o == -2 ? 1.f : o == -1 ? -8.f : o == 0 ? 0.f : o == 1 ? 8.f : -1.f;
            const float ca = o == -2 ? -1.f : o == -1 ? 16.f : o == 0 ? -30.f : o == 1 ? 16.f : -1.f;
            const float cj = o == -2 ? -1.f : o == -1 ? 2.f : o == 0 ? 0.f : o == 1 ? -2.f : 1.f;
            g += sd[0] * cv * inv12dt + sd[1] * ca * inv12dt2 + sd[2] * cj * inv2dt3;
          }
        }
      }
      if (a.grad) a.grad[vbase + k] = g;
    }

    // per-state world and self costs (optional output)
    if (a.state_terms) {
      float2* out = reinterpret_cast<float2*>(a.state_terms) + vbase / D;
      for (int k = tid; k < S; k += nthr) out[k] = make_float2(s_stw[k], selfc ? prm.w_self * s_sts[k] : 0.f);
    }
    // ---- per-trajectory cost in a fixed order, from the last warp down (the
    // first warps still hold gradient items of this pass)
    for (int r = nw - 1 - warp; r >= 0 && r < nt; r += nw) {
      float tw = 0.f, ts = 0.f, tb = 0.f, tsm = 0.f;
      for (int t = lane; t < H; t += 32) {
        tw += s_stw[r * H + t];
        if (selfc) ts += prm.w_self * s_sts[r * H + t];
      }
      for (int k = lane; k < H * D; k += 32) tb += s_pb[r * H * D + k];
      if (!ik) {
        for (int k = lane; k < NS * D; k += 32) {
          tb += s_db[r * NS * D + k];
          tsm += s_sm[r * NS * D + k];
        }
      }
      tw = warp_sum(tw);
      ts = warp_sum(ts);
      tb = warp_sum(tb);
      tsm = warp_sum(tsm);
      if (lane == 0) {
        const int gi = s_prob.traj_base + r0 + r;
        const float tg = s_goal[r];
        a.cost[gi] = tw + ts + tb + tsm + tg;
        if (a.cfree) a.cfree[gi] = (uint8_t)(s_free[r] != 0);
        if (a.terms) {
          float* tt = a.terms + (long long)gi * CR_N_TERMS;
          tt[0] = tw;
          tt[1] = ts;
          tt[2] = tb;
          tt[3] = tsm;
          tt[4] = tg;
        }
      }
    }
    if (a.queue) {
      __syncthreads();
      if (tid == 0) s_next = atomicAdd(a.queue, 1);
      __syncthreads();
      tile = s_next;
    } else {
      tile += gridDim.x;
    }
  }
}

// Forward kinematics of N configurations, one thread each.
__global__ void k_fk(RobotView rb, const float* __restrict__ theta, int n, float* spheres, float* ee,
                     float* link_tf) {
  __shared__ float s_fix[(kMaxDof + 1) * 12];
  __shared__ int s_axis[kMaxDof];
  const int D = rb.dof;
  for (int k = threadIdx.x; k < (D + 1) * 12; k += blockDim.x) s_fix[k] = rb.fixed_tf[k];
  for (int k = threadIdx.x; k < D; k += blockDim.x) s_axis[k] = rb.axis[k];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float q[kMaxDof];
  for (int j = 0; j < D; ++j) q[j] = theta[(long long)b * D + j];
  alignas(16) float LT[kMaxDof * 12];
  fk_chain(s_fix, s_axis, D, q, nullptr, LT);
  if (link_tf)
    for (int k = 0; k < D * 12; ++k) link_tf[(long long)b * D * 12 + k] = LT[k];
  if (ee) {
    const float* T6 = LT + (D - 1) * 12;
    const float* Fe = s_fix + D * 12;
    for (int rr = 0; rr < 3; ++rr)
      for (int cc = 0; cc < 4; ++cc) {
        float v = fmaf(T6[4 * rr], Fe[cc], fmaf(T6[4 * rr + 1], Fe[4 + cc], T6[4 * rr + 2] * Fe[8 + cc]));
        ee[(long long)b * 12 + 4 * rr + cc] = cc == 3 ? v + T6[4 * rr + 3] : v;
      }
  }
  if (spheres) {
    for (int i = 0; i < rb.n_spheres; ++i) {
      const float4 c = rb.spheres[i];
      const V3 x = tf_point(LT + rb.sphere_link[i] * 12, c.x, c.y, c.z);
      reinterpret_cast<float4*>(spheres)[(long long)b * rb.n_spheres + i] = make_float4(x.x, x.y, x.z, c.w);
    }
  }
}

}  // namespace

// The largest dynamic shared memory any launch may ask for (the opt-in
// limit) is set once per device, never lowered, so launches captured in a
// graph stay valid whatever is launched later.
template <int MinBlocks>
static cudaError_t allow_smem(int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_eval<MinBlocks>);
  if (e != cudaSuccess) return e;
  // opt-in limit minus the kernel's static shared memory
  return cudaFuncSetAttribute(k_eval<MinBlocks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

cudaError_t allow_eval_smem() {
  static unsigned done = 0;  // bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  if (done & bit) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = allow_smem<1>(optin);
  if (e == cudaSuccess) e = allow_smem<2>(optin);
  if (e == cudaSuccess) done |= bit;
  return e;
}

int eval_smem_limit() {
  static int cached[32] = {};  // per device
  int dev = 0;
  cudaGetDevice(&dev);
  int& c = cached[dev & 31];
  if (c == 0) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    c = optin - 1024;  // room for the kernel's static shared memory
  }
  return c;
}

// Kernel variant and layout of a launch.  no_store_x = 1 takes the
// two-CTAs-per-SM variant without the position cache; 0 the one-CTA variant,
// positions cached in shared memory when they fit; -1 (auto) the first when
// two of its CTAs fit on an SM, else the second.
static EvalSmem eval_layout(const EvalArgs& a, int block, bool* store_x, bool* two) {
  EvalSmem L;
  int mode = a.no_store_x;
  if (mode < 0) {
    L.build(a.rb.dof, a.rb.n_spheres, a.rb.n_pairs, a.rb.n_groups, a.max_traj, a.max_states,
            block / 32, false);
    int n = 0;
    allow_eval_smem();
    if (L.bytes <= eval_smem_limit() &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval<2>, block, L.bytes) != cudaSuccess)
      n = 0;
    mode = n >= 2 ? 1 : 0;
  }
  *two = mode == 1;
  L.build(a.rb.dof, a.rb.n_spheres, a.rb.n_pairs, a.rb.n_groups, a.max_traj, a.max_states,
          block / 32, true);
  *store_x = mode == 0 && L.bytes <= eval_smem_limit();
  if (!*store_x)
    L.build(a.rb.dof, a.rb.n_spheres, a.rb.n_pairs, a.rb.n_groups, a.max_traj, a.max_states,
            block / 32, false);
  return L;
}

int eval_smem_bytes(const EvalArgs& a, int block) {
  if (a.prm.flags & CR_IK_MODE) return eval_ik_smem_bytes(a.rb.dof);
  bool sx, two;
  return eval_layout(a, block, &sx, &two).bytes;
}

int eval_blocks_per_sm(const EvalArgs& a, int block) {
  if (a.prm.flags & CR_IK_MODE) return eval_ik_blocks_per_sm(a.rb.dof);
  bool sx, two;
  const int smem = eval_layout(a, block, &sx, &two).bytes;
  int n = 0;
  allow_eval_smem();
  if (two)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval<2>, block, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval<1>, block, smem);
  return n;
}

cudaError_t launch_eval(const EvalArgs& a_in, int grid, int block, cudaStream_t stream) {
  if (a_in.prm.flags & CR_IK_MODE) return launch_eval_ik(a_in, stream);
  EvalArgs a = a_in;
  bool sx, two;
  const int smem = eval_layout(a, block, &sx, &two).bytes;
  a.store_x = sx ? 1 : 0;
  cudaError_t e = allow_eval_smem();
  if (e != cudaSuccess) return e;
  return two ? launch_pdl(k_eval<2>, grid, block, smem, stream, a)
             : launch_pdl(k_eval<1>, grid, block, smem, stream, a);
}

cudaError_t launch_fk(const RobotView& rb, const float* theta, int n, float* spheres, float* ee,
                      float* link_tf, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int block = 128;
  k_fk<<<(n + block - 1) / block, block, 0, stream>>>(rb, theta, n, spheres, ee, link_tf);
  return cudaGetLastError();
}

}  // namespace crgb
