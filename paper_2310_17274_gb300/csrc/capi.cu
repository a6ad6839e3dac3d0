// capi.cu -- the C ABI of include/crgb.h: handles, validation, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "crgb_internal.cuh"

using namespace crgb;

namespace {

thread_local std::string g_err;

cr_status fail(cr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

cr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CR_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

}  // namespace

cr_status crgb::set_error(cr_status code, const char* msg) {
  g_err = msg;
  return code;
}

extern "C" {

const char* cr_last_error(void) { return g_err.c_str(); }

const char* cr_version(void) { return "crgb 0.1 (sm_103a)"; }

void cr_params_default(cr_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->w_goal_pos = 2000.f;  // App. A.1: alpha_0..alpha_3
  p->w_goal_rot = 350.f;
  p->k_goal_pos = 100.f;
  p->k_goal_rot = 100.f;
  p->w_coll = 5000.f;      // App. B.3: weight 5000 for soft constraints
  p->w_self = 5000.f;
  p->w_bound = 5000.f;
  p->w_acc = 5000.f;       // App. A.2: alpha_8, alpha_9, alpha_6, alpha_7
  p->w_jerk = 1.f;
  p->w_vel = 5000.f;
  p->k_vel = 50.f;
  p->eta = 0.025f;         // App. B.3: 2.5 cm
  p->eta_bound = 0.1f;     // App. A.3
  p->dt = 0.05f;
  p->sweep_steps = 4;
  p->history = 6;
  p->n_alpha = 4;          // Sec. 7.3 noisy-ls step sizes
  p->alpha[0] = 0.01f;
  p->alpha[1] = 0.3f;
  p->alpha[2] = 0.7f;
  p->alpha[3] = 1.0f;
  p->armijo_c1 = 1e-4f;
  p->wolfe_c2 = 0.9f;
  p->flags = CR_SWEPT | CR_SPEED | CR_SELF | CR_WOLFE;
  p->w_cspace = 5000.f;  // alpha_4, App. A.1 (Eq. 15)
  p->k_cspace = 50.f;    // alpha_5
}

cr_status cr_robot_create(const cr_robot_desc* d, cr_robot** out) {
  if (!d || !out) return fail(CR_EINVAL, "cr_robot_create: null argument");
  *out = nullptr;
  const int D = d->dof, M = d->n_spheres, P = d->n_pairs;
  if (D < 1 || D > kMaxDof) return fail(CR_EINVAL, "dof %d outside 1..%d", D, kMaxDof);
  if (M < 1 || M > kMaxSpheres) return fail(CR_EINVAL, "n_spheres %d outside 1..%d", M, kMaxSpheres);
  if (P < 0 || P > kMaxPairs) return fail(CR_EINVAL, "n_pairs %d outside 0..%d", P, kMaxPairs);
  if (!d->fixed_tf || !d->axis || !d->q_lo || !d->q_hi || !d->v_max || !d->a_max || !d->j_max ||
      !d->spheres || !d->sphere_link || (P > 0 && !d->pairs))
    return fail(CR_EINVAL, "cr_robot_create: null array");
  for (int j = 0; j < D; ++j) {
    if (d->axis[j] < 0 || d->axis[j] > 2) return fail(CR_EINVAL, "axis[%d] = %d not in 0..2", j, d->axis[j]);
    if (!(d->q_lo[j] < d->q_hi[j])) return fail(CR_EINVAL, "q_lo[%d] >= q_hi[%d]", j, j);
    if (!(d->v_max[j] > 0 && d->a_max[j] > 0 && d->j_max[j] > 0))
      return fail(CR_EINVAL, "derivative limits of joint %d must be > 0", j);
  }
  for (int i = 0; i < M; ++i)
    if (d->sphere_link[i] < 0 || d->sphere_link[i] >= D)
      return fail(CR_EINVAL, "sphere_link[%d] = %d not in 0..%d", i, d->sphere_link[i], D - 1);
  for (int p = 0; p < P; ++p) {
    int i = d->pairs[2 * p], j = d->pairs[2 * p + 1];
    if (i < 0 || i >= M || j < 0 || j >= M || i == j)
      return fail(CR_EINVAL, "pair %d = (%d, %d) invalid", p, i, j);
  }
  // Bounding sphere of each link's enabled spheres (link frame): a lower
  // bound on every distance of the link's spheres, used to skip whole links.
  std::vector<float> lbs((size_t)D * 4, 0.f), soff(M, 0.f), ldmax(D, 0.f);
  for (int l = 0; l < D; ++l) {
    double c[3] = {0, 0, 0};
    int cnt = 0;
    for (int i = 0; i < M; ++i)
      if (d->sphere_link[i] == l && d->spheres[4 * i + 3] >= 0.f) {
        for (int a = 0; a < 3; ++a) c[a] += d->spheres[4 * i + a];
        ++cnt;
      }
    double R = -1.0;
    if (cnt > 0) {
      for (int a = 0; a < 3; ++a) c[a] /= cnt;
      for (int i = 0; i < M; ++i)
        if (d->sphere_link[i] == l && d->spheres[4 * i + 3] >= 0.f) {
          double dx = d->spheres[4 * i] - c[0], dy = d->spheres[4 * i + 1] - c[1],
                 dz = d->spheres[4 * i + 2] - c[2];
          double o = std::sqrt(dx * dx + dy * dy + dz * dz);
          soff[i] = (float)(o * (1.0 + 1e-6) + 1e-6);  // rounded up: stays a bound in FP32
          R = std::max(R, (double)soff[i] + d->spheres[4 * i + 3]);
          ldmax[l] = std::max(ldmax[l], soff[i]);
        }
    }
    for (int a = 0; a < 3; ++a) lbs[4 * l + a] = (float)c[a];
    lbs[4 * l + 3] = (float)R;
  }
  // pairs grouped by link pair (stable), keeping each pair's original position
  std::vector<int> order(P);
  for (int p = 0; p < P; ++p) order[p] = p;
  auto key = [&](int p) {
    int a = d->sphere_link[d->pairs[2 * p]], b = d->sphere_link[d->pairs[2 * p + 1]];
    return std::min(a, b) * kMaxDof + std::max(a, b);
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
  std::vector<uint32_t> pairs(P);
  std::vector<int> orig(P);
  std::vector<int4> groups;
  for (int q = 0; q < P; ++q) {
    const int p = order[q];
    pairs[q] = (uint32_t)d->pairs[2 * p] | ((uint32_t)d->pairs[2 * p + 1] << 16);
    orig[q] = p;
    const int k = key(p);
    if (groups.empty() || key(order[groups.back().z]) != k)
      groups.push_back(make_int4(k / kMaxDof, k % kMaxDof, q, 0));
    groups.back().w += 1;
  }
  const int G = (int)groups.size();
  // spheres by link (ascending index within a link)
  std::vector<int> lstart(D + 1, 0), lsph(M > 0 ? M : 1);
  int max_ls = 0;
  for (int i = 0; i < M; ++i) lstart[d->sphere_link[i] + 1] += 1;
  for (int l = 0; l < D; ++l) {
    max_ls = std::max(max_ls, lstart[l + 1]);
    lstart[l + 1] += lstart[l];
  }
  {
    std::vector<int> fill(lstart.begin(), lstart.end() - 1);
    for (int i = 0; i < M; ++i) lsph[fill[d->sphere_link[i]]++] = i;
  }
  // robots of up to 64 spheres: the grouped index of the pair {i, j} at [i][j]
  // and [j][i] (the caller's first when listed twice), -1 when not a pair
  const int n_at = M <= kPairTableSpheres && P <= 32767 ? M * M : 0;
  std::vector<int16_t> pair_at((size_t)(n_at > 0 ? n_at : 1), (int16_t)-1);
  for (int q = 0; q < P && n_at > 0; ++q) {
    const int i = (int)(pairs[q] & 0xffffu), j = (int)(pairs[q] >> 16);
    for (int side = 0; side < 2; ++side) {
      int16_t& at = side == 0 ? pair_at[(size_t)i * M + j] : pair_at[(size_t)j * M + i];
      if (at < 0 || orig[q] < orig[at]) at = (int16_t)q;
    }
  }
  // one blob: fixed_tf | lim | spheres (float4) | axis | link | offsets | link spheres | pairs |
  // original positions | groups | pair table
  const size_t n_fix = (size_t)(D + 1) * 12, n_lim = (size_t)5 * D;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = (off + bytes + 255) & ~size_t(255); return r; };
  const size_t o_fix = take(n_fix * 4), o_lim = take(n_lim * 4), o_sph = take((size_t)M * 16),
               o_axis = take((size_t)D * 4), o_link = take((size_t)M * 4),
               o_soff = take((size_t)M * 4), o_lbs = take((size_t)D * 16), o_ldm = take((size_t)D * 4),
               o_pairs = take((size_t)(P > 0 ? P : 1) * 4), o_orig = take((size_t)(P > 0 ? P : 1) * 4),
               o_grp = take((size_t)(G > 0 ? G : 1) * 16), o_lst = take((size_t)(D + 1) * 4),
               o_lsp = take((size_t)(M > 0 ? M : 1) * 4), o_pat = take(pair_at.size() * 2),
               o_ls4 = take((size_t)(M > 0 ? M : 1) * 16);
  std::vector<unsigned char> host(off, 0);
  std::memcpy(host.data() + o_fix, d->fixed_tf, n_fix * 4);
  float* lim = reinterpret_cast<float*>(host.data() + o_lim);
  for (int j = 0; j < D; ++j) {
    lim[j] = d->q_lo[j];
    lim[D + j] = d->q_hi[j];
    lim[2 * D + j] = d->v_max[j];
    lim[3 * D + j] = d->a_max[j];
    lim[4 * D + j] = d->j_max[j];
  }
  std::memcpy(host.data() + o_sph, d->spheres, (size_t)M * 16);
  std::memcpy(host.data() + o_axis, d->axis, (size_t)D * 4);
  std::memcpy(host.data() + o_link, d->sphere_link, (size_t)M * 4);
  std::memcpy(host.data() + o_soff, soff.data(), (size_t)M * 4);
  std::memcpy(host.data() + o_lbs, lbs.data(), (size_t)D * 16);
  std::memcpy(host.data() + o_ldm, ldmax.data(), (size_t)D * 4);
  if (P > 0) {
    std::memcpy(host.data() + o_pairs, pairs.data(), (size_t)P * 4);
    std::memcpy(host.data() + o_orig, orig.data(), (size_t)P * 4);
  }
  if (G > 0) std::memcpy(host.data() + o_grp, groups.data(), (size_t)G * 16);
  std::memcpy(host.data() + o_lst, lstart.data(), (size_t)(D + 1) * 4);
  std::memcpy(host.data() + o_lsp, lsph.data(), (size_t)M * 4);
  std::memcpy(host.data() + o_pat, pair_at.data(), pair_at.size() * 2);
  for (int q = 0; q < M; ++q) std::memcpy(host.data() + o_ls4 + (size_t)q * 16, d->spheres + 4 * lsph[q], 16);
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, off);
  if (e != cudaSuccess) return fail(CR_ENOMEM, "cudaMalloc(%zu): %s", off, cudaGetErrorString(e));
  e = cudaMemcpy(dev, host.data(), off, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "cudaMemcpy(robot)");
  }
  cr_robot* r = new cr_robot();
  r->dof = D;
  r->n_spheres = M;
  r->n_pairs = P;
  r->dev = dev;
  unsigned char* b = static_cast<unsigned char*>(dev);
  r->view.dof = D;
  r->view.n_spheres = M;
  r->view.n_pairs = P;
  r->view.fixed_tf = reinterpret_cast<const float*>(b + o_fix);
  r->view.lim = reinterpret_cast<const float*>(b + o_lim);
  r->view.spheres = reinterpret_cast<const float4*>(b + o_sph);
  r->view.axis = reinterpret_cast<const int*>(b + o_axis);
  r->view.sphere_link = reinterpret_cast<const int*>(b + o_link);
  r->view.pairs = reinterpret_cast<const uint32_t*>(b + o_pairs);
  r->view.pair_orig = reinterpret_cast<const int*>(b + o_orig);
  r->view.groups = reinterpret_cast<const int4*>(b + o_grp);
  r->view.n_groups = G;
  r->view.sphere_off = reinterpret_cast<const float*>(b + o_soff);
  r->view.link_bs = reinterpret_cast<const float4*>(b + o_lbs);
  r->view.link_dmax = reinterpret_cast<const float*>(b + o_ldm);
  r->view.link_start = reinterpret_cast<const int*>(b + o_lst);
  r->view.link_sph = reinterpret_cast<const int*>(b + o_lsp);
  r->view.max_link_spheres = max_ls;
  r->view.fd_dof = make_fastdiv(D);
  r->view.fd_sph = make_fastdiv(M);
  r->view.fd_grp = make_fastdiv(G);
  r->view.fd_lsph = make_fastdiv(max_ls);
  r->view.pair_at = n_at > 0 ? reinterpret_cast<const int16_t*>(b + o_pat) : nullptr;
  r->view.link_sph4 = reinterpret_cast<const float4*>(b + o_ls4);
  for (int j = 0; j < D; ++j) {
    r->q_lo[j] = d->q_lo[j];
    r->q_hi[j] = d->q_hi[j];
  }
  *out = r;
  return CR_OK;
}

void cr_robot_destroy(cr_robot* r) {
  if (!r) return;
  cudaFree(r->dev);
  delete r;
}

// rotation (row-major) of a quaternion wxyz, normalised; false if degenerate
static bool quat_rot(const float* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  if (!(n > 1e-12) || !std::isfinite(n)) return false;
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
  return true;
}

cr_status cr_world_create(const cr_world_desc* d, cr_world** out) {
  if (!d || !out) return fail(CR_EINVAL, "cr_world_create: null argument");
  *out = nullptr;
  if (d->n < 0 || d->n > kMaxBoxes) return fail(CR_EINVAL, "n boxes %d outside 0..%d", d->n, kMaxBoxes);
  if (d->n > 0 && (!d->pose || !d->half_ext)) return fail(CR_EINVAL, "cr_world_create: null array");
  std::vector<BoxRows> rows((size_t)(d->n > 0 ? d->n : 1));
  for (int k = 0; k < d->n; ++k) {
    const float* p = d->pose + 7 * k;
    const float* h = d->half_ext + 3 * k;
    double R[9];
    if (!quat_rot(p + 3, R)) return fail(CR_EINVAL, "box %d: degenerate quaternion", k);
    if (!(h[0] > 0 && h[1] > 0 && h[2] > 0)) return fail(CR_EINVAL, "box %d: half extents must be > 0", k);
    // u = R^T (x - c) = R^T x + t, t = -R^T c
    float4* r = &rows[k].r0;
    for (int a = 0; a < 3; ++a) {
      double t = -(R[0 * 3 + a] * p[0] + R[1 * 3 + a] * p[1] + R[2 * 3 + a] * p[2]);
      r[a] = make_float4((float)R[0 * 3 + a], (float)R[1 * 3 + a], (float)R[2 * 3 + a], (float)t);
    }
    const float hn = (float)std::sqrt((double)h[0] * h[0] + (double)h[1] * h[1] + (double)h[2] * h[2]);
    rows[k].h = make_float4(h[0], h[1], h[2], hn);
    rows[k].c = make_float4(p[0], p[1], p[2], hn);
  }
  BoxRows* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, rows.size() * sizeof(BoxRows));
  if (e != cudaSuccess) return fail(CR_ENOMEM, "cudaMalloc(world): %s", cudaGetErrorString(e));
  e = cudaMemcpy(dev, rows.data(), rows.size() * sizeof(BoxRows), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "cudaMemcpy(world)");
  }
  cr_world* w = new cr_world();
  w->n = d->n;
  w->dev = dev;
  *out = w;
  return CR_OK;
}

void cr_world_destroy(cr_world* w) {
  if (!w) return;
  cudaFree(w->dev);
  delete w;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// shared checks and argument builders
// ---------------------------------------------------------------------------

namespace crgb {

cr_status check_params(const cr_params* p) {
  if (!p) return fail(CR_EINVAL, "null params");
  if (p->history < 1 || p->history > CR_MAX_HISTORY)
    return fail(CR_EINVAL, "history %d outside 1..%d", p->history, CR_MAX_HISTORY);
  if (p->n_alpha < 1 || p->n_alpha > CR_MAX_ALPHA)
    return fail(CR_EINVAL, "n_alpha %d outside 1..%d", p->n_alpha, CR_MAX_ALPHA);
  if (!(p->eta > 0) || !(p->eta_bound > 0) || !(p->dt > 0))
    return fail(CR_EINVAL, "eta, eta_bound and dt must be > 0");
  if (p->sweep_steps < 0 || p->sweep_steps > 64) return fail(CR_EINVAL, "sweep_steps outside 0..64");
  if ((p->flags & CR_NO_SELF_CHECK) && (!(p->flags & CR_IK_MODE) || (p->flags & CR_SELF)))
    return fail(CR_EINVAL, "CR_NO_SELF_CHECK needs CR_IK_MODE without CR_SELF");
  return CR_OK;
}

cr_status fill_problem(const cr_robot* rb, const cr_problem* pr, ProblemView* pv, const cr_params* prm) {
  if (!pr || !pr->world || !pr->q_start || !pr->goal) return fail(CR_EINVAL, "problem: null field");
  if (pr->horizon < 1 || pr->horizon > kMaxHorizon)
    return fail(CR_EINVAL, "horizon %d outside 1..%d", pr->horizon, kMaxHorizon);
  std::memset(pv, 0, sizeof(*pv));
  pv->boxes = pr->world->dev;
  pv->n_boxes = pr->world->n;
  pv->horizon = pr->horizon;
  pv->fd_h = make_fastdiv(pr->horizon);
  pv->fd_hd = make_fastdiv((pr->horizon + 1) * rb->dof);
  for (int j = 0; j < rb->dof; ++j) pv->q_start[j] = pr->q_start[j];
  for (int a = 0; a < 3; ++a) pv->goal_p[a] = pr->goal[a];
  double R[9];
  if (!quat_rot(pr->goal + 3, R)) return fail(CR_EINVAL, "goal: degenerate quaternion");
  for (int k = 0; k < 9; ++k) pv->goal_R[k] = (float)R[k];
  if (pr->goal_q) {
    pv->has_goal_q = 1;
    for (int j = 0; j < rb->dof; ++j) pv->goal_q[j] = pr->goal_q[j];
  }
  if (prm) {
    pv->dt = prm->dt;
    pv->w_vel = prm->w_vel;
    pv->w_acc = prm->w_acc;
    pv->w_jerk = prm->w_jerk;
  }
  return CR_OK;
}

}  // namespace crgb

extern "C" {

cr_status cr_fk(const cr_robot* robot, const float* theta, int32_t n, float* spheres, float* ee,
                float* link_tf, void* stream) {
  if (!robot || (n > 0 && !theta)) return fail(CR_EINVAL, "cr_fk: null argument");
  if (n < 0) return fail(CR_EINVAL, "cr_fk: n < 0");
  cudaError_t e = launch_fk(robot->view, theta, n, spheres, ee, link_tf, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cr_fk launch");
  return CR_OK;
}

cr_status cr_eval(const cr_robot* robot, const cr_problem* problem, const cr_params* params,
                  const float* theta, int32_t B, float* cost, float* grad, uint8_t* cfree,
                  float* terms, float* state_terms, void* stream) {
  if (!robot) return fail(CR_EINVAL, "cr_eval: null robot");
  cr_status s = check_params(params);
  if (s != CR_OK) return s;
  if (B < 0) return fail(CR_EINVAL, "cr_eval: B < 0");
  if (B > 0 && (!theta || !cost)) return fail(CR_EINVAL, "cr_eval: null theta or cost");
  EvalArgs a{};
  std::memset(&a, 0, sizeof(a));
  s = fill_problem(robot, problem, &a.prob0, params);
  if (s != CR_OK) return s;
  if (B == 0) return CR_OK;
  const int H = problem->horizon;
  a.rb = robot->view;
  a.prm = *params;
  a.prob0.n_traj = B;
  a.problems = nullptr;
  a.traj_per_tile = H >= 32 ? 1 : (32 + H - 1) / H;
  if (a.traj_per_tile > B) a.traj_per_tile = B;
  a.max_traj = a.traj_per_tile;
  a.max_states = a.traj_per_tile * H;
  a.max_horizon = H;
  a.theta = theta;
  a.cost = cost;
  a.grad = grad;
  a.cfree = cfree;
  a.terms = terms;
  a.state_terms = state_terms;
  a.no_store_x = -1;
  const int block = kEvalBlock;
  const int smem = eval_smem_bytes(a, block);
  if (smem > eval_smem_limit())
    return fail(CR_EINVAL, "cr_eval: tile needs %d bytes of shared memory (> 227 KB)", smem);
  const int grid = (B + a.traj_per_tile - 1) / a.traj_per_tile;
  cudaError_t e = launch_eval(a, grid, block, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cr_eval launch");
  return CR_OK;
}

static cr_status opt_common(const cr_robot* robot, const cr_params* params, const cr_opt_state* st,
                            OptArgs* a) {
  cr_status s = check_params(params);
  if (s != CR_OK) return s;
  if (!st) return fail(CR_EINVAL, "null optimiser state");
  if (st->n_seeds < 0 || st->horizon < 1 || st->horizon > kMaxHorizon)
    return fail(CR_EINVAL, "optimiser state: bad n_seeds / horizon");
  std::memset(a, 0, sizeof(*a));
  a->prm = *params;
  a->st = *st;
  a->n_seeds = st->n_seeds;
  a->horizon = st->horizon;
  a->dof = robot ? robot->dof : 0;
  return CR_OK;
}

cr_status cr_opt_propose(const cr_robot* robot, const cr_params* params, const cr_opt_state* st,
                         void* stream) {
  if (!robot) return fail(CR_EINVAL, "cr_opt_propose: null robot");
  OptArgs a{};
  cr_status s = opt_common(robot, params, st, &a);
  if (s != CR_OK) return s;
  const int n = st->horizon * robot->dof;
  if (n > 2048) return fail(CR_EINVAL, "horizon * dof = %d > 2048", n);
  if (opt_smem_bytes(params->history, n) > 200 * 1024)
    return fail(CR_EINVAL, "history * horizon * dof too large for shared memory");
  a.q_lo = robot->view.lim;
  a.q_hi = robot->view.lim + robot->dof;
  a.do_propose = 1;
  cudaError_t e = launch_opt(a, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cr_opt_propose launch");
  return CR_OK;
}

cr_status cr_opt_select(const cr_robot* robot, const cr_params* params, const cr_opt_state* st,
                        void* stream) {
  if (!robot) return fail(CR_EINVAL, "cr_opt_select: null robot");
  OptArgs a{};
  cr_status s = opt_common(robot, params, st, &a);
  if (s != CR_OK) return s;
  const int n = st->horizon * robot->dof;
  if (n > 2048) return fail(CR_EINVAL, "horizon * dof = %d > 2048", n);
  a.do_select = 1;
  cudaError_t e = launch_opt(a, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cr_opt_select launch");
  return CR_OK;
}

}  // extern "C"
