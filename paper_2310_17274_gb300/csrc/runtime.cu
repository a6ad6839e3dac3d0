// runtime.cu -- context, workspace and the batched, graph-captured solve of
// many uneven problems (Sec. 4.1: iterations of L-BFGS + parallel noisy line
// search with best-iterate tracking; App. D: iterations captured in a CUDA
// graph).
//
// Layout of a batch of P problems (problem p: B_p seeds, horizon H_p, n_p =
// H_p * dof variables per seed): per-seed arrays are concatenated problem by
// problem, so seed b of problem p starts at float offset vo_p + b n_p; the
// n_alpha line-search candidates of a seed are contiguous ([B_p][n_alpha][n_p]
// per problem).  One evaluation launch covers every problem: a tile table
// lists (problem, first trajectory, count) and CTAs take tiles from a device
// counter, largest tiles first.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "crgb_internal.cuh"

using namespace crgb;

namespace crgb {
cr_status check_params(const cr_params* p);
}  // namespace crgb

namespace {

cr_status failf(cr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define RT_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return failf(CR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Best seed per problem: the lowest-cost collision-free seed, else the
// lowest-cost seed (App. A.9 picks among valid seeds); copy out every seed's
// best iterate, cost and flag.
__global__ void k_finish(const ResultView* res, int n_problems, const float* best_x,
                         const float* best_c, const uint8_t* best_cfree) {
  const int p = blockIdx.x;
  if (p >= n_problems) return;
  const ResultView r = res[p];
  __shared__ int s_best;
  if (threadIdx.x == 0) {
    int bi = 0, bf = -1;
    float bc = INFINITY, fc = INFINITY;
    bool finite = true;
    for (int b = 0; b < r.n_seeds; ++b) {
      const float c = best_c[r.seed_base + b];
      finite = finite && isfinite(c);
      if (c < bc) {
        bc = c;
        bi = b;
      }
      if (best_cfree[r.seed_base + b] && (bf < 0 || c < fc)) {
        fc = c;
        bf = b;
      }
    }
    s_best = bf >= 0 ? bf : bi;
    if (r.best) *r.best = s_best;
    // a seed whose best cost is not finite (a non-finite seed, or an overflow)
    if (r.status) *r.status = finite ? CR_OK : CR_ENAN;
  }
  __syncthreads();
  const long long total = (long long)r.n_seeds * r.n;
  if (r.traj)
    for (long long k = threadIdx.x; k < total; k += blockDim.x) r.traj[k] = best_x[r.var_base + k];
  for (int b = threadIdx.x; b < r.n_seeds; b += blockDim.x) {
    if (r.cost) r.cost[b] = best_c[r.seed_base + b];
    if (r.cfree) r.cfree[b] = best_cfree[r.seed_base + b];
  }
}

}  // namespace

cudaError_t crgb::launch_finish(const ResultView* res, int n_problems, const float* best_x,
                                const float* best_c, const uint8_t* best_cfree, cudaStream_t s) {
  if (n_problems <= 0) return cudaSuccess;
  k_finish<<<n_problems, 256, 0, s>>>(res, n_problems, best_x, best_c, best_cfree);
  return cudaGetLastError();
}

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

// Plan of one batch: tables, workspace carve-up and launch shapes.
struct Plan {
  int P = 0, S = 0, dof = 0, m = 0, na = 0;
  long long V = 0;
  int n_max = 0;
  std::vector<ProblemView> probs_x, probs_c, probs_p;
  std::vector<int4> tiles_x, tiles_c, tiles_p, seedtab;
  int max_traj_p = 0, max_states_p = 0, n_part = 0;
  std::vector<ResultView> results;
  int max_traj_x = 0, max_states_x = 0, max_traj_c = 0, max_states_c = 0, max_h = 0;
  int block = kEvalBlock;
  int no_store_x = 0;
  // workspace offsets (bytes)
  size_t o_x, o_g, o_xp, o_gp, o_dir, o_bx, o_c, o_bc, o_rho, o_it, o_s, o_y, o_cand, o_cgrad,
      o_ccost, o_cfree, o_bfree, o_ls, o_queue, o_tdt, o_tsc, o_sig, o_part, o_pcost, ws_bytes;
  size_t o_tx, o_tc, o_px, o_pc, o_seed, o_res, o_tv, o_tp, o_pp, tab_bytes;
};

// Particle-based optimisation of every seed before L-BFGS (Sec. 4.2, App.
// B.3: two iterations for IK and trajectory optimisation).
struct ParticlePlan {
  cr_particle_config cfg;
};

// A time-discretised solve (Alg. "Time Discretization"): two solves with the
// device steps of k_time.cu between and after them.
struct TimeoptPlan {
  TimeScale sc;
  int iters1 = 0, iters2 = 0;
  std::vector<TimeoptView> views;
};

struct cr_ctx {
  int device = 0;
  size_t mem_budget = 0;
  int n_sm = 0;
  cudaStream_t cap = nullptr;
  DevBuf ws, tab;
  std::vector<unsigned char> tab_host;
  unsigned char* tab_pinned = nullptr;
  size_t tab_pinned_bytes = 0;
  cudaEvent_t staged = nullptr;  // recorded after the last copy out of tab_pinned
  // graph cache: key bytes -> executable graph
  std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;
  // autotune table: (spheres, box-count bucket, horizon) -> (CTA threads,
  // states per tile for horizons below 32)
  std::map<long long, int4> tune;  // (block, short_tile, no position cache, -)
  ~cr_ctx() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    if (cap) cudaStreamDestroy(cap);
    if (tab_pinned) cudaFreeHost(tab_pinned);
    if (staged) cudaEventDestroy(staged);
  }
};

namespace {

// Tile shape of a problem: whole trajectories per tile; horizons below 32
// pack ceil(short_tile / H) trajectories so a tile holds about short_tile states.
int traj_per_tile(int H, int short_tile = 32) { return H >= 32 ? 1 : (short_tile + H - 1) / H; }

int pow2_bucket(int K) {
  int b = 1;
  while (b < K) b <<= 1;
  return b;
}

long long tune_key(int M, int K, int H) { return ((long long)M << 40) | ((long long)pow2_bucket(K) << 16) | H; }

// tuned (block, short_tile, no position cache) for a problem shape, else the defaults
int4 tuned(const cr_ctx* ctx, int M, int K, int H) {
  auto it = ctx->tune.find(tune_key(M, K, H));
  if (it != ctx->tune.end()) return it->second;
  return make_int4(kEvalBlock, 32, -1, 0);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

cr_status build_plan(cr_ctx* ctx, const cr_robot* rb, int P, const cr_problem* pr,
                     const cr_params* prm, const cr_result* res, const TimeoptPlan* to,
                     const ParticlePlan* pp, Plan& pl) {
  pl.P = P;
  pl.n_part = pp ? pp->cfg.n_particles : 0;
  pl.dof = rb->dof;
  pl.m = prm->history;
  pl.na = prm->n_alpha;
  pl.probs_x.resize(P);
  pl.probs_c.resize(P);
  pl.results.resize(P);
  long long vo = 0;
  int sb = 0;
  for (int p = 0; p < P; ++p) {
    if (pr[p].n_seeds < 1) return failf(CR_EINVAL, "problem %d: n_seeds < 1", p);
    ProblemView pv;
    cr_status s = fill_problem(rb, &pr[p], &pv, prm);
    if (s != CR_OK) return s;
    const int H = pr[p].horizon, B = pr[p].n_seeds, n = H * rb->dof;
    if (n > 2048) return failf(CR_EINVAL, "problem %d: horizon * dof = %d > 2048", p, n);
    pl.n_max = std::max(pl.n_max, n);
    pl.max_h = std::max(pl.max_h, H);
    pv.n_traj = B;
    pv.traj_base = sb;
    pv.var_base = vo;
    pl.probs_x[p] = pv;
    ProblemView pc = pv;
    pc.n_traj = B * pl.na;
    pc.traj_base = sb * pl.na;
    pc.var_base = vo * pl.na;
    pl.probs_c[p] = pc;
    if (pl.n_part > 0) {  // the particles of every seed, [B][n_particles][n] per problem
      ProblemView pq = pv;
      pq.n_traj = B * pl.n_part;
      pq.traj_base = sb * pl.n_part;
      pq.var_base = vo * pl.n_part;
      pl.probs_p.push_back(pq);
    }
    for (int b = 0; b < B; ++b) pl.seedtab.push_back(make_int4(n, (int)(vo + (long long)b * n), sb + b, p));
    ResultView rv;
    rv.traj = res ? res[p].traj : nullptr;
    rv.cost = res ? res[p].cost : nullptr;
    rv.cfree = res ? res[p].cfree : nullptr;
    rv.best = res ? res[p].best : nullptr;
    rv.status = res ? res[p].status : nullptr;
    rv.n_seeds = B;
    rv.n = n;
    rv.seed_base = sb;
    rv.var_base = (int)vo;
    pl.results[p] = rv;
    vo += (long long)B * n;
    sb += B;
  }
  pl.S = sb;
  pl.V = vo;
  const int4 tc = tuned(ctx, rb->n_spheres, pr[0].world->n, pr[0].horizon);
  pl.block = tc.x;
  pl.no_store_x = tc.z;
  if (pl.V * pl.na > (1ll << 31) - 1) return failf(CR_EINVAL, "batch too large");
  // tiles, largest first (cost ~ states x boxes), so a counter-driven
  // persistent launch ends with small tiles
  auto make_tiles = [&](const std::vector<ProblemView>& pvs, std::vector<int4>& tiles, int& mt,
                        int& ms) {
    std::vector<std::pair<long long, int4>> tmp;
    for (int p = 0; p < P; ++p) {
      const int H = pvs[p].horizon;
      const int nt = traj_per_tile(H, tuned(ctx, rb->n_spheres, pvs[p].n_boxes, H).y);
      for (int r0 = 0; r0 < pvs[p].n_traj; r0 += nt) {
        const int c = std::min(nt, pvs[p].n_traj - r0);
        tmp.push_back({(long long)c * H * (pvs[p].n_boxes + 8), make_int4(p, r0, c, 0)});
        mt = std::max(mt, c);
        ms = std::max(ms, c * H);
      }
    }
    std::stable_sort(tmp.begin(), tmp.end(),
                     [](const std::pair<long long, int4>& a, const std::pair<long long, int4>& b) {
                       return a.first > b.first;
                     });
    tiles.clear();
    for (auto& t : tmp) tiles.push_back(t.second);
  };
  make_tiles(pl.probs_x, pl.tiles_x, pl.max_traj_x, pl.max_states_x);
  make_tiles(pl.probs_c, pl.tiles_c, pl.max_traj_c, pl.max_states_c);
  if (pl.n_part > 0) {
    if (pl.V * pl.n_part > (1ll << 31) - 1) return failf(CR_EINVAL, "batch too large for its particles");
    make_tiles(pl.probs_p, pl.tiles_p, pl.max_traj_p, pl.max_states_p);
  }
  // workspace
  const size_t V = (size_t)pl.V, S = (size_t)pl.S, m = pl.m, na = pl.na;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  pl.o_x = take(V * 4); pl.o_g = take(V * 4); pl.o_xp = take(V * 4); pl.o_gp = take(V * 4);
  pl.o_dir = take(V * 4); pl.o_bx = take(V * 4); pl.o_c = take(S * 4); pl.o_bc = take(S * 4);
  pl.o_rho = take(S * m * 4); pl.o_it = take(S * 4); pl.o_s = take(V * m * 4);
  pl.o_y = take(V * m * 4); pl.o_cand = take(V * na * 4); pl.o_cgrad = take(V * na * 4);
  pl.o_ccost = take(S * na * 4); pl.o_cfree = take(S * na); pl.o_bfree = take(S);
  pl.o_ls = take(S * 4); pl.o_queue = take(256);
  pl.o_tdt = take(to ? S * 4 : 0); pl.o_tsc = take(to ? S * 4 : 0);
  const size_t np = (size_t)pl.n_part;
  pl.o_sig = take(np ? V * 4 : 0); pl.o_part = take(V * np * 4); pl.o_pcost = take(S * np * 4);
  pl.ws_bytes = o;
  o = 0;
  pl.o_tx = take(pl.tiles_x.size() * sizeof(int4));
  pl.o_tc = take(pl.tiles_c.size() * sizeof(int4));
  pl.o_px = take(P * sizeof(ProblemView));
  pl.o_pc = take(P * sizeof(ProblemView));
  pl.o_seed = take(pl.seedtab.size() * sizeof(int4));
  pl.o_res = take(P * sizeof(ResultView));
  pl.o_tv = take(to ? P * sizeof(TimeoptView) : 0);
  pl.o_tp = take(pl.tiles_p.size() * sizeof(int4));
  pl.o_pp = take(pl.probs_p.size() * sizeof(ProblemView));
  pl.tab_bytes = o;
  if (ctx->mem_budget && pl.ws_bytes + pl.tab_bytes > ctx->mem_budget)
    return failf(CR_ENOMEM, "batch needs %zu bytes > context budget %zu", pl.ws_bytes + pl.tab_bytes,
                 ctx->mem_budget);
  return CR_OK;
}

cr_opt_state state_of(const Plan& pl, unsigned char* ws) {
  cr_opt_state st;
  std::memset(&st, 0, sizeof(st));
  st.n_seeds = pl.S;
  st.horizon = 0;
  st.x = (float*)(ws + pl.o_x);
  st.g = (float*)(ws + pl.o_g);
  st.c = (float*)(ws + pl.o_c);
  st.x_prev = (float*)(ws + pl.o_xp);
  st.g_prev = (float*)(ws + pl.o_gp);
  st.s = (float*)(ws + pl.o_s);
  st.y = (float*)(ws + pl.o_y);
  st.rho = (float*)(ws + pl.o_rho);
  st.iter = (int32_t*)(ws + pl.o_it);
  st.dir = (float*)(ws + pl.o_dir);
  st.cand = (float*)(ws + pl.o_cand);
  st.cand_cost = (float*)(ws + pl.o_ccost);
  st.cand_grad = (float*)(ws + pl.o_cgrad);
  st.cand_cfree = (uint8_t*)(ws + pl.o_cfree);
  st.best_x = (float*)(ws + pl.o_bx);
  st.best_c = (float*)(ws + pl.o_bc);
  st.best_cfree = (uint8_t*)(ws + pl.o_bfree);
  st.ls_index = (int32_t*)(ws + pl.o_ls);
  return st;
}

// Enqueue the iterations on `s` (eagerly or under capture); with `finish`
// the per-problem results are written at the end.
cr_status enqueue_iterations(cr_ctx* ctx, const cr_robot* rb, const cr_params* prm, const Plan& pl,
                             unsigned char* ws, unsigned char* tab, int iters, bool persistent,
                             cudaStream_t s, bool finish = true, const ParticlePlan* pp = nullptr) {
  const cr_opt_state st = state_of(pl, ws);
  int* queue = (int*)(ws + pl.o_queue);
  auto eval_args = [&](bool cand) {
    EvalArgs a{};
    std::memset(&a, 0, sizeof(a));
    a.rb = rb->view;
    a.prm = *prm;
    a.problems = (const ProblemView*)(tab + (cand ? pl.o_pc : pl.o_px));
    a.tiles = (const int4*)(tab + (cand ? pl.o_tc : pl.o_tx));
    a.n_tiles = (int)(cand ? pl.tiles_c.size() : pl.tiles_x.size());
    a.max_traj = cand ? pl.max_traj_c : pl.max_traj_x;
    a.max_states = cand ? pl.max_states_c : pl.max_states_x;
    a.max_horizon = pl.max_h;
    a.theta = cand ? st.cand : st.x;
    a.cost = cand ? st.cand_cost : st.c;
    a.grad = cand ? st.cand_grad : st.g;
    a.cfree = cand ? st.cand_cfree : st.best_cfree;
    a.terms = nullptr;
    a.queue = nullptr;
    a.no_store_x = pl.no_store_x;
    return a;
  };
  // Persistent form: a grid of resident CTAs taking tiles from a device
  // counter, used when there are more tiles than resident CTAs (the counter
  // then balances uneven tiles); with fewer, one CTA per tile is cheaper.
  // The counter is zeroed before the first evaluation and by every optimiser
  // launch after the evaluation it follows.
  auto launch_eval_batch = [&](bool cand) -> cr_status {
    EvalArgs a = eval_args(cand);
    const int block = pl.block;
    const int smem = eval_smem_bytes(a, block);
    if (smem > eval_smem_limit()) return failf(CR_EINVAL, "tile needs %d bytes of shared memory", smem);
    int grid = a.n_tiles;
    if (persistent) {
      const int per_sm = std::max(1, eval_blocks_per_sm(a, block));
      if (a.n_tiles > per_sm * ctx->n_sm) {
        grid = per_sm * ctx->n_sm;
        a.queue = queue;
      }
    }
    RT_CUDA(launch_eval(a, grid, block, s));
    return CR_OK;
  };
  OptArgs o{};
  std::memset(&o, 0, sizeof(o));
  o.prm = *prm;
  o.q_lo = rb->view.lim;
  o.q_hi = rb->view.lim + rb->dof;
  o.dof = rb->dof;
  o.n_seeds = pl.S;
  o.seed_tab = (const int4*)(tab + pl.o_seed);
  o.st = st;
  o.reset_queue = persistent ? queue : nullptr;

  // particle-based optimisation (Sec. 4.2) moves every seed first: the seeds
  // are the means, sigma0 the initial variance; per iteration the samples,
  // their costs (one evaluation launch over every particle of every problem,
  // no gradients) and the update of mean and variance
  if (pp && pp->cfg.iters > 0) {
    const cr_particle_config& c = pp->cfg;
    float* sigma = (float*)(ws + pl.o_sig);
    float* part = (float*)(ws + pl.o_part);
    float* pcost = (float*)(ws + pl.o_pcost);
    const int4* seeds = (const int4*)(tab + pl.o_seed);
    RT_CUDA(launch_fill(sigma, pl.V, c.sigma0, s));
    for (int k = 0; k < c.iters; ++k) {
      const float* eps = c.eps + (size_t)k * c.n_particles * pl.V;
      RT_CUDA(launch_particle_batch(seeds, pl.S, c.n_particles, 0, eps, st.x, sigma, part, nullptr, c.beta, c.k_mu,
                                    c.k_sigma, s));
      EvalArgs a{};
      std::memset(&a, 0, sizeof(a));
      a.rb = rb->view;
      a.prm = *prm;
      a.problems = (const ProblemView*)(tab + pl.o_pp);
      a.tiles = (const int4*)(tab + pl.o_tp);
      a.n_tiles = (int)pl.tiles_p.size();
      a.max_traj = pl.max_traj_p;
      a.max_states = pl.max_states_p;
      a.max_horizon = pl.max_h;
      a.theta = part;
      a.cost = pcost;
      a.no_store_x = pl.no_store_x;
      const int smem = eval_smem_bytes(a, pl.block);
      if (smem > eval_smem_limit()) return failf(CR_EINVAL, "particle tile needs %d bytes of shared memory", smem);
      int grid = a.n_tiles;
      const int per_sm = std::max(1, eval_blocks_per_sm(a, pl.block));
      if (a.n_tiles > per_sm * ctx->n_sm) {
        grid = per_sm * ctx->n_sm;
        a.queue = queue;
        RT_CUDA(cudaMemsetAsync(queue, 0, sizeof(int), s));
      }
      RT_CUDA(launch_eval(a, grid, pl.block, s));
      RT_CUDA(launch_particle_batch(seeds, pl.S, c.n_particles, 1, nullptr, st.x, sigma, part, pcost, c.beta,
                                    c.k_mu, c.k_sigma, s));
    }
  }
  // iteration state starts empty
  RT_CUDA(cudaMemsetAsync(st.s, 0, (size_t)pl.V * pl.m * 4, s));
  RT_CUDA(cudaMemsetAsync(st.y, 0, (size_t)pl.V * pl.m * 4, s));
  RT_CUDA(cudaMemsetAsync(st.rho, 0, (size_t)pl.S * pl.m * 4, s));
  RT_CUDA(cudaMemsetAsync(st.iter, 0, (size_t)pl.S * 4, s));
  if (persistent) RT_CUDA(cudaMemsetAsync(queue, 0, sizeof(int), s));
  cr_status rs = launch_eval_batch(false);
  if (rs != CR_OK) return rs;
  o.init_best = 1;
  o.do_propose = iters > 0;
  RT_CUDA(launch_opt(o, pl.n_max, s));
  o.init_best = 0;
  for (int it = 0; it < iters; ++it) {
    rs = launch_eval_batch(true);
    if (rs != CR_OK) return rs;
    o.do_select = 1;
    o.do_propose = it + 1 < iters;
    o.early_loads = 1;  // follows the candidate evaluation directly
    RT_CUDA(launch_opt(o, pl.n_max, s));
  }
  if (finish)
    RT_CUDA(launch_finish((const ResultView*)(tab + pl.o_res), pl.P, st.best_x, st.best_c,
                          st.best_cfree, s));
  return CR_OK;
}

// Alg. "Time Discretization" on `s`: the first solve (the tables hold the
// first step and weights), the device step that retimes each problem's best
// seed and rewrites the tables for the second solve, the second solve from
// every seed's best iterate, then every seed retimed, scored and chosen.
cr_status enqueue_timeopt(cr_ctx* ctx, const cr_robot* rb, const cr_params* prm, const Plan& pl,
                          const TimeoptPlan& to, unsigned char* ws, unsigned char* tab, bool persistent,
                          cudaStream_t s) {
  const cr_opt_state st = state_of(pl, ws);
  const TimeoptView* tv = (const TimeoptView*)(tab + pl.o_tv);
  cr_status rs = enqueue_iterations(ctx, rb, prm, pl, ws, tab, to.iters1, persistent, s, false);
  if (rs != CR_OK) return rs;
  RT_CUDA(launch_timeopt_mid((ProblemView*)(tab + pl.o_px), (ProblemView*)(tab + pl.o_pc), pl.P, tv, rb->view,
                             st.best_x, st.best_c, st.best_cfree, st.x, to.sc, s));
  rs = enqueue_iterations(ctx, rb, prm, pl, ws, tab, to.iters2, persistent, s, true);
  if (rs != CR_OK) return rs;
  RT_CUDA(launch_timeopt_final((const ProblemView*)(tab + pl.o_px), pl.P, tv, rb->view, st.best_x, st.best_c,
                               st.best_cfree, (float*)(ws + pl.o_tdt), (float*)(ws + pl.o_tsc), to.sc, s));
  return CR_OK;
}

std::string graph_key(const cr_robot* rb, const cr_params* prm, const Plan& pl, int iters,
                      bool persistent, const void* ws, const void* tab, int block, const TimeoptPlan* to,
                      const ParticlePlan* pp) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  const int kind = (to ? 1 : 0) | (pp ? 2 : 0);
  put(&kind, sizeof(kind));
  if (pp) put(&pp->cfg, sizeof(pp->cfg));  // the samples' address included
  if (to) {
    put(&to->sc, sizeof(to->sc));
    put(&to->iters1, sizeof(int));
    put(&to->iters2, sizeof(int));
  }
  put(&rb, sizeof(rb));
  put(prm, sizeof(*prm));
  put(&iters, sizeof(iters));
  put(&persistent, sizeof(persistent));
  put(&ws, sizeof(ws));
  put(&tab, sizeof(tab));
  put(&block, sizeof(block));
  put(&pl.P, sizeof(int));
  const int nts[3] = {(int)pl.tiles_x.size(), (int)pl.tiles_c.size(), pl.no_store_x};
  put(nts, sizeof(nts));
  for (int p = 0; p < pl.P; ++p) {
    int shp[3] = {pl.probs_x[p].n_traj, pl.probs_x[p].horizon, pl.probs_x[p].n_boxes};
    put(shp, sizeof(shp));
  }
  return k;
}

}  // namespace

extern "C" {

cr_status cr_context_create(int device, size_t mem_budget, cr_ctx** out) {
  if (!out) return failf(CR_EINVAL, "cr_context_create: null out");
  *out = nullptr;
  int n = 0;
  RT_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return failf(CR_EINVAL, "device %d not in 0..%d", device, n - 1);
  RT_CUDA(cudaSetDevice(device));
  cr_ctx* c = new cr_ctx();
  c->device = device;
  c->mem_budget = mem_budget;
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return failf(CR_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
  }
  *out = c;
  return CR_OK;
}

void cr_context_destroy(cr_ctx* c) { delete c; }

}  // extern "C"

namespace {

// The body of cr_solve and cr_solve_timeopt (to != nullptr).
cr_status solve_impl(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                     const cr_params* params, int32_t iters, uint32_t solve_flags, const cr_result* results,
                     void* stream, const TimeoptPlan* to, const ParticlePlan* pp = nullptr) {
  if (!ctx || !robot || !problems || n_problems < 1) return failf(CR_EINVAL, "cr_solve: bad argument");
  if (iters < 0) return failf(CR_EINVAL, "cr_solve: iters < 0");
  cr_status s = check_params(params);
  if (s != CR_OK) return s;
  for (int p = 0; p < n_problems; ++p)
    if (!problems[p].seeds) return failf(CR_EINVAL, "problem %d: null seeds", p);
  Plan pl;
  s = build_plan(ctx, robot, n_problems, problems, params, results, to, pp, pl);
  if (s != CR_OK) return s;
  if (opt_smem_bytes(params->history, pl.n_max) > 200 * 1024)
    return failf(CR_EINVAL, "history * horizon * dof too large for shared memory");
  cudaStream_t st = (cudaStream_t)stream;
  // a new workspace or table address invalidates the cached graphs
  const void* ws0 = ctx->ws.p;
  const void* tab0 = ctx->tab.p;
  cudaError_t e = ctx->ws.ensure(pl.ws_bytes);
  if (e != cudaSuccess) return failf(CR_ENOMEM, "workspace of %zu bytes: %s", pl.ws_bytes, cudaGetErrorString(e));
  e = ctx->tab.ensure(pl.tab_bytes);
  if (e != cudaSuccess) return failf(CR_ENOMEM, "tables of %zu bytes: %s", pl.tab_bytes, cudaGetErrorString(e));
  if (ws0 != ctx->ws.p || tab0 != ctx->tab.p) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
  }
  unsigned char* ws = (unsigned char*)ctx->ws.p;
  unsigned char* tab = (unsigned char*)ctx->tab.p;
  // tables through a pinned staging buffer; the previous call's copy out of
  // it must have finished before it is rewritten
  if (ctx->staged) RT_CUDA(cudaEventSynchronize(ctx->staged));
  // host seeds are gathered behind the tables and copied in one piece (the x
  // region holds the problems' seeds back to back)
  const bool host_seeds = !(solve_flags & CR_SOLVE_DEVICE_SEEDS);
  const size_t seed_off = (pl.tab_bytes + 255) & ~size_t(255);
  const size_t staged_bytes = host_seeds ? seed_off + (size_t)pl.V * 4 : pl.tab_bytes;
  if (ctx->tab_pinned_bytes < staged_bytes) {
    if (ctx->tab_pinned) cudaFreeHost(ctx->tab_pinned);
    ctx->tab_pinned = nullptr;
    ctx->tab_pinned_bytes = 0;
    RT_CUDA(cudaMallocHost(&ctx->tab_pinned, staged_bytes));
    ctx->tab_pinned_bytes = staged_bytes;
  }
  if (!ctx->staged) RT_CUDA(cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming));
  unsigned char* h = ctx->tab_pinned;
  std::memcpy(h + pl.o_tx, pl.tiles_x.data(), pl.tiles_x.size() * sizeof(int4));
  std::memcpy(h + pl.o_tc, pl.tiles_c.data(), pl.tiles_c.size() * sizeof(int4));
  std::memcpy(h + pl.o_px, pl.probs_x.data(), pl.P * sizeof(ProblemView));
  std::memcpy(h + pl.o_pc, pl.probs_c.data(), pl.P * sizeof(ProblemView));
  std::memcpy(h + pl.o_seed, pl.seedtab.data(), pl.seedtab.size() * sizeof(int4));
  std::memcpy(h + pl.o_res, pl.results.data(), pl.P * sizeof(ResultView));
  if (to) std::memcpy(h + pl.o_tv, to->views.data(), pl.P * sizeof(TimeoptView));
  if (!pl.tiles_p.empty()) std::memcpy(h + pl.o_tp, pl.tiles_p.data(), pl.tiles_p.size() * sizeof(int4));
  if (!pl.probs_p.empty()) std::memcpy(h + pl.o_pp, pl.probs_p.data(), pl.probs_p.size() * sizeof(ProblemView));
  RT_CUDA(cudaMemcpyAsync(tab, h, pl.tab_bytes, cudaMemcpyHostToDevice, st));
  // seeds -> x (host memory, or device memory with CR_SOLVE_DEVICE_SEEDS)
  if (host_seeds) {
    for (int p = 0; p < n_problems; ++p) {
      const size_t bytes = (size_t)problems[p].n_seeds * problems[p].horizon * robot->dof * 4;
      std::memcpy(h + seed_off + (size_t)pl.probs_x[p].var_base * 4, problems[p].seeds, bytes);
    }
    RT_CUDA(cudaMemcpyAsync(ws + pl.o_x, h + seed_off, (size_t)pl.V * 4, cudaMemcpyHostToDevice, st));
  } else {
    for (int p = 0; p < n_problems; ++p) {
      const size_t bytes = (size_t)problems[p].n_seeds * problems[p].horizon * robot->dof * 4;
      RT_CUDA(cudaMemcpyAsync(ws + pl.o_x + (size_t)pl.probs_x[p].var_base * 4, problems[p].seeds, bytes,
                              cudaMemcpyDeviceToDevice, st));
    }
  }
  RT_CUDA(cudaEventRecord(ctx->staged, st));
  const bool persistent = (solve_flags & CR_SOLVE_PERSISTENT) != 0;
  auto enqueue = [&](cudaStream_t q) {
    return to ? enqueue_timeopt(ctx, robot, params, pl, *to, ws, tab, persistent, q)
              : enqueue_iterations(ctx, robot, params, pl, ws, tab, iters, persistent, q, true, pp);
  };
  if (!(solve_flags & CR_SOLVE_GRAPH)) return enqueue(st);
  const std::string key = graph_key(robot, params, pl, iters, persistent, ws, tab, pl.block, to, pp);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : ctx->graphs)
    if (g.first == key) exec = g.second;
  if (!exec) {
    // capture on the context's stream, ordered after the copies on `st`
    cudaEvent_t ev;
    RT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    RT_CUDA(cudaEventRecord(ev, st));
    RT_CUDA(cudaStreamWaitEvent(ctx->cap, ev, 0));
    cudaEventDestroy(ev);
    RT_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cr_status cs = enqueue(ctx->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
    if (cs != CR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return cs;
    }
    if (ce != cudaSuccess) return failf(CR_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return failf(CR_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ce));
    if (ctx->graphs.size() >= 8) {
      cudaGraphExecDestroy(ctx->graphs.front().second);
      ctx->graphs.erase(ctx->graphs.begin());
    }
    ctx->graphs.push_back({key, exec});
  }
  RT_CUDA(cudaGraphLaunch(exec, st));
  return CR_OK;
}

}  // namespace

extern "C" {

cr_status cr_solve(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                   const cr_params* params, int32_t iters, uint32_t solve_flags,
                   const cr_result* results, void* stream) {
  return solve_impl(ctx, robot, n_problems, problems, params, iters, solve_flags, results, stream, nullptr);
}

cr_status cr_solve_particles(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                             const cr_params* params, int32_t iters, uint32_t solve_flags,
                             const cr_particle_config* particles, const cr_result* results, void* stream) {
  if (!particles) return failf(CR_EINVAL, "cr_solve_particles: null particle configuration");
  const cr_particle_config& c = *particles;
  if (c.iters < 0 || c.n_particles < 1 || c.n_particles > 4096)
    return failf(CR_EINVAL, "cr_solve_particles: iters < 0 or n_particles outside 1..4096");
  if (!(c.beta > 0.f) || !(c.k_mu >= 0.f && c.k_mu <= 1.f) || !(c.k_sigma >= 0.f && c.k_sigma <= 1.f) ||
      !(c.sigma0 >= 0.f))
    return failf(CR_EINVAL, "cr_solve_particles: beta must be > 0, k_mu and k_sigma in [0, 1], sigma0 >= 0");
  if (c.iters > 0 && !c.eps) return failf(CR_EINVAL, "cr_solve_particles: null samples");
  ParticlePlan pp;
  pp.cfg = c;
  return solve_impl(ctx, robot, n_problems, problems, params, iters, solve_flags, results, stream, nullptr, &pp);
}

cr_status cr_solve_timeopt(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems, const cr_problem* problems,
                           const cr_params* params, const cr_timeopt_config* cfg, uint32_t solve_flags,
                           const cr_result* results, const cr_timeopt_result* tres, void* stream) {
  if (!cfg) return failf(CR_EINVAL, "cr_solve_timeopt: null config");
  cr_status s = check_params(params);
  if (s != CR_OK) return s;
  if (params->flags & CR_IK_MODE) return failf(CR_EINVAL, "cr_solve_timeopt: not for IK-mode problems");
  if (!(cfg->dt_init > 0.f) || !(cfg->dt_min > 0.f))
    return failf(CR_EINVAL, "cr_solve_timeopt: dt_init and dt_min must be > 0");
  if (cfg->iters1 < 0 || cfg->iters2 < 0) return failf(CR_EINVAL, "cr_solve_timeopt: iterations < 0");
  TimeoptPlan to;
  to.sc.dt0 = params->dt;
  to.sc.w_vel0 = params->w_vel;
  to.sc.w_acc0 = params->w_acc;
  to.sc.w_jerk0 = params->w_jerk;
  to.sc.dt_min = cfg->dt_min;
  to.sc.rank_pose = cfg->w_pose;
  to.sc.rank_jerk = cfg->w_jerk;
  to.sc.rank_time = cfg->w_time;
  to.iters1 = cfg->iters1;
  to.iters2 = cfg->iters2;
  to.views.resize(n_problems > 0 ? n_problems : 0);
  for (int p = 0; p < n_problems; ++p) {
    TimeoptView v{};
    if (tres) {
      v.first = tres[p].first;
      v.stage = tres[p].stage;
      v.dt = tres[p].dt;
      v.score = tres[p].score;
      v.chosen = tres[p].chosen;
    }
    to.views[p] = v;
  }
  // the first solve's step and weights (no jerk term) go into the tables
  cr_params p1 = *params;
  float w1[4];
  time_scaled(to.sc, cfg->dt_init, false, w1);
  p1.dt = w1[0];
  p1.w_vel = w1[1];
  p1.w_acc = w1[2];
  p1.w_jerk = w1[3];
  return solve_impl(ctx, robot, n_problems, problems, &p1, cfg->iters1 + cfg->iters2, solve_flags, results,
                    stream, &to);
}

}  // extern "C"

extern "C" cr_status cr_autotune(cr_ctx* ctx, const cr_robot* robot, int32_t n_problems,
                                 const cr_problem* problems, const cr_params* params, int32_t iters,
                                 int32_t* block_out, int32_t* short_tile_out, int32_t* no_cache_out,
                                 float* ms_out) {
  if (!ctx || !robot || !problems || n_problems < 1) return failf(CR_EINVAL, "cr_autotune: bad argument");
  if (iters < 1) iters = 2;
  int min_h = kMaxHorizon;
  for (int p = 0; p < n_problems; ++p) min_h = std::min(min_h, problems[p].horizon);
  const int blocks[2] = {256, 512};
  std::vector<int> shorts = {32};
  if (min_h < 32) shorts = {8, 16, 32, 64};
  const int caches[2] = {0, 1};
  cudaStream_t s = nullptr;
  RT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  RT_CUDA(cudaEventCreate(&e0));
  RT_CUDA(cudaEventCreate(&e1));
  // results go to scratch outputs owned by the context workspace: none needed
  float best_ms = INFINITY;
  int4 best = make_int4(kEvalBlock, 32, 0, 0);
  const std::map<long long, int4> saved = ctx->tune;
  cr_status st = CR_OK;
  for (int bl : blocks) {
    for (int sh : shorts)
    for (int nc : caches) {
      for (int p = 0; p < n_problems; ++p)
        ctx->tune[tune_key(robot->n_spheres, problems[p].world->n, problems[p].horizon)] = make_int4(bl, sh, nc, 0);
      // warm-up, then timed
      st = cr_solve(ctx, robot, n_problems, problems, params, iters, CR_SOLVE_PERSISTENT, nullptr, s);
      if (st != CR_OK) break;
      RT_CUDA(cudaEventRecord(e0, s));
      st = cr_solve(ctx, robot, n_problems, problems, params, iters, CR_SOLVE_PERSISTENT, nullptr, s);
      if (st != CR_OK) break;
      RT_CUDA(cudaEventRecord(e1, s));
      RT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      RT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = make_int4(bl, sh, nc, 0);
      }
    }
    if (st != CR_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  ctx->tune = saved;
  if (st != CR_OK) return st;
  for (int p = 0; p < n_problems; ++p)
    ctx->tune[tune_key(robot->n_spheres, problems[p].world->n, problems[p].horizon)] = best;
  if (block_out) *block_out = best.x;
  if (short_tile_out) *short_tile_out = best.y;
  if (no_cache_out) *no_cache_out = best.z;
  if (ms_out) *ms_out = best_ms;
  return CR_OK;
}

extern "C" cr_status cr_tune_set(cr_ctx* ctx, int32_t n_spheres, int32_t n_boxes, int32_t horizon,
                                 int32_t block, int32_t short_tile, int32_t no_cache) {
  if (!ctx) return failf(CR_EINVAL, "cr_tune_set: null context");
  if (block != 256 && block != 512) return failf(CR_EINVAL, "cr_tune_set: block must be 256 or 512");
  if (short_tile < 1 || short_tile > 128) return failf(CR_EINVAL, "cr_tune_set: short_tile outside 1..128");
  ctx->tune[tune_key(n_spheres, n_boxes, horizon)] = make_int4(block, short_tile, no_cache < 0 ? -1 : (no_cache ? 1 : 0), 0);
  return CR_OK;
}
