// server.cu -- continuous batching of motion-generation and IK requests
// with device-resident optimiser state and admission by free device memory.
//
// Requests of two kinds (0: trajectory optimisation / motion generation,
// 1: IK) each have a fixed shape per kind (seeds, horizon, iterations,
// parameters).  A kind keeps a pool of request slots: every per-seed array
// of the optimiser (iterate, gradient, history, candidates, best iterate) is
// one device array with room for `capacity` slots, slot s owning seeds
// s*B .. s*B + B - 1.  A step (cr_server_step)
//   1. admits queued requests into free slots, growing a pool (doubling, the
//      live slots copied over) only while free device memory minus the
//      reserve allows, and runs their initial evaluation + first L-BFGS step;
//   2. runs `chunk` iterations (one evaluation launch over the line-search
//      candidates of every active request of the kind, one selection + L-BFGS
//      launch over their seeds) for all active requests, the two kinds on
//      two streams so their kernels overlap;
//   3. retires requests that reached their iteration count: best seed per
//      request, results copied to host, slot freed.
// A request's arithmetic never depends on the other requests, so its result
// is bit-identical to cr_solve of that request alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "crgb_internal.cuh"

using namespace crgb;

namespace {

cr_status failf(cr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define SV_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return failf(CR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Result staging of one slot: traj [B][n] | cost [B] | cfree [B] | best.
struct ResLayout {
  size_t cost, cfree, best, bytes;
  ResLayout(int B, int n) {
    cost = (size_t)B * n * 4;
    cfree = cost + (size_t)B * 4;
    best = (cfree + B + 3) & ~size_t(3);
    bytes = a256(best + 4);
  }
};

int traj_per_tile(int H) { return H >= 32 ? 1 : (32 + H - 1) / H; }

struct Request {
  uint64_t ticket = 0;
  int kind = 0;
  const cr_world* world = nullptr;
  std::vector<float> q_start, goal, seeds;
  int slot = -1;
  int iters_done = 0;
  bool done = false;
  std::vector<float> traj, cost;
  std::vector<uint8_t> cfree;
  int best = -1;
};

// Field-major device pool of one request kind.
struct Pool {
  int kind = 0;
  int B = 0, H = 0, n = 0, m = 0, na = 0, iters = 0;
  cr_params prm{};
  int capacity = 0;
  void* base = nullptr;
  size_t bytes = 0;
  // field offsets (bytes) for the current capacity
  size_t o_x, o_g, o_xp, o_gp, o_dir, o_bx, o_c, o_bc, o_rho, o_it, o_s, o_y, o_cand, o_cgrad,
      o_ccost, o_cfree, o_bfree, o_ls, o_queue, o_res;
  std::vector<int> slot_req;  // request index per slot, -1 free
  // per-step tables
  void* tab = nullptr;
  size_t tab_bytes = 0;
  unsigned char* tab_host = nullptr;
  size_t tab_host_bytes = 0;
  // result staging (device) for retiring slots
  cudaStream_t stream = nullptr;

  // carve-up for `cap` slots; returns total bytes
  size_t layout(int cap, Pool* out) const {
    const size_t S = (size_t)cap * B, V = S * n;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o = a256(o + b); return r; };
    size_t f[20];
    f[0] = take(V * 4); f[1] = take(V * 4); f[2] = take(V * 4); f[3] = take(V * 4);
    f[4] = take(V * 4); f[5] = take(V * 4); f[6] = take(S * 4); f[7] = take(S * 4);
    f[8] = take(S * m * 4); f[9] = take(S * 4); f[10] = take(V * m * 4); f[11] = take(V * m * 4);
    f[12] = take(V * na * 4); f[13] = take(V * na * 4); f[14] = take(S * na * 4);
    f[15] = take(S * na); f[16] = take(S); f[17] = take(S * 4); f[18] = take(256);
    f[19] = take((size_t)cap * ResLayout(B, n).bytes);  // result staging
    if (out) {
      out->o_x = f[0]; out->o_g = f[1]; out->o_xp = f[2]; out->o_gp = f[3]; out->o_dir = f[4];
      out->o_bx = f[5]; out->o_c = f[6]; out->o_bc = f[7]; out->o_rho = f[8]; out->o_it = f[9];
      out->o_s = f[10]; out->o_y = f[11]; out->o_cand = f[12]; out->o_cgrad = f[13];
      out->o_ccost = f[14]; out->o_cfree = f[15]; out->o_bfree = f[16]; out->o_ls = f[17];
      out->o_queue = f[18]; out->o_res = f[19];
    }
    return o;
  }

  unsigned char* p(size_t off) const { return static_cast<unsigned char*>(base) + off; }

  cr_opt_state state() const {
    cr_opt_state st;
    std::memset(&st, 0, sizeof(st));
    st.n_seeds = capacity * B;
    st.horizon = H;
    st.x = (float*)p(o_x); st.g = (float*)p(o_g); st.c = (float*)p(o_c);
    st.x_prev = (float*)p(o_xp); st.g_prev = (float*)p(o_gp);
    st.s = (float*)p(o_s); st.y = (float*)p(o_y); st.rho = (float*)p(o_rho);
    st.iter = (int32_t*)p(o_it); st.dir = (float*)p(o_dir); st.cand = (float*)p(o_cand);
    st.cand_cost = (float*)p(o_ccost); st.cand_grad = (float*)p(o_cgrad);
    st.cand_cfree = (uint8_t*)p(o_cfree); st.best_x = (float*)p(o_bx); st.best_c = (float*)p(o_bc);
    st.best_cfree = (uint8_t*)p(o_bfree); st.ls_index = (int32_t*)p(o_ls);
    return st;
  }
};

}  // namespace

struct cr_server {
  cr_ctx* ctx = nullptr;
  const cr_robot* robot = nullptr;
  cr_server_config cfg{};
  Pool pool[2];
  std::vector<std::unique_ptr<Request>> reqs;  // every submitted request
  std::map<uint64_t, size_t> by_ticket;
  std::deque<size_t> queue;                    // waiting for a slot
  uint64_t next_ticket = 1;
  int n_sm = 0;
  ~cr_server() {
    for (auto& pl : pool) {
      if (pl.base) cudaFree(pl.base);
      if (pl.tab) cudaFree(pl.tab);
      if (pl.tab_host) cudaFreeHost(pl.tab_host);
      if (pl.stream) cudaStreamDestroy(pl.stream);
    }
  }
};

namespace {

// Grow a pool to `cap` slots when free memory minus the reserve allows,
// copying the live slots' state (field by field) into the new arrays.
cr_status grow(cr_server* sv, Pool& pl, int cap, bool* grown) {
  *grown = false;
  Pool nl = pl;
  const size_t need = pl.layout(cap, &nl);
  size_t free_b = 0, total_b = 0;
  SV_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t extra = need > pl.bytes ? need - pl.bytes : 0;
  if (free_b < sv->cfg.reserve_bytes || free_b - sv->cfg.reserve_bytes < extra) return CR_OK;
  void* nb = nullptr;
  if (cudaMalloc(&nb, need) != cudaSuccess) {
    cudaGetLastError();
    return CR_OK;  // refused: requests keep waiting
  }
  nl.base = nb;
  nl.bytes = need;
  nl.capacity = cap;
  if (pl.base) {
    SV_CUDA(cudaStreamSynchronize(pl.stream));
    const size_t S0 = (size_t)pl.capacity * pl.B, V0 = S0 * pl.n;
    const size_t sizes[18] = {V0 * 4, V0 * 4, V0 * 4, V0 * 4, V0 * 4, V0 * 4, S0 * 4, S0 * 4,
                              S0 * pl.m * 4, S0 * 4, V0 * pl.m * 4, V0 * pl.m * 4, V0 * pl.na * 4,
                              V0 * pl.na * 4, S0 * pl.na * 4, S0 * pl.na, S0, S0 * 4};
    const size_t from[18] = {pl.o_x, pl.o_g, pl.o_xp, pl.o_gp, pl.o_dir, pl.o_bx, pl.o_c, pl.o_bc,
                             pl.o_rho, pl.o_it, pl.o_s, pl.o_y, pl.o_cand, pl.o_cgrad, pl.o_ccost,
                             pl.o_cfree, pl.o_bfree, pl.o_ls};
    const size_t to[18] = {nl.o_x, nl.o_g, nl.o_xp, nl.o_gp, nl.o_dir, nl.o_bx, nl.o_c, nl.o_bc,
                           nl.o_rho, nl.o_it, nl.o_s, nl.o_y, nl.o_cand, nl.o_cgrad, nl.o_ccost,
                           nl.o_cfree, nl.o_bfree, nl.o_ls};
    for (int f = 0; f < 18; ++f)
      SV_CUDA(cudaMemcpyAsync(nl.p(to[f]), pl.p(from[f]), sizes[f], cudaMemcpyDeviceToDevice, pl.stream));
    SV_CUDA(cudaStreamSynchronize(pl.stream));
    cudaFree(pl.base);
  }
  nl.slot_req.resize(cap, -1);
  pl = nl;
  *grown = true;
  return CR_OK;
}

int free_slot(const Pool& pl) {
  for (int s = 0; s < pl.capacity; ++s)
    if (pl.slot_req[s] < 0) return s;
  return -1;
}

// Tables of one launch round for a set of slots: problem views for the
// iterate (x) or candidate evaluation, tiles, seed table, result views.
struct Tables {
  std::vector<ProblemView> px, pc;
  std::vector<int4> tx, tc, seeds;
  std::vector<ResultView> res;
};

cr_status slot_view(cr_server* sv, Pool& pl, int s, const Request& r, ProblemView* v) {
  cr_problem pr;
  std::memset(&pr, 0, sizeof(pr));
  pr.world = r.world;
  pr.q_start = r.q_start.data();
  pr.goal = r.goal.data();
  pr.n_seeds = pl.B;
  pr.horizon = pl.H;
  cr_status st = fill_problem(sv->robot, &pr, v, &pl.prm);
  if (st != CR_OK) return st;
  v->n_traj = pl.B;
  v->traj_base = s * pl.B;
  v->var_base = (long long)s * pl.B * pl.n;
  return CR_OK;
}

void add_tiles(std::vector<int4>& tiles, int p, int n_traj, int H) {
  const int nt = traj_per_tile(H);
  for (int r0 = 0; r0 < n_traj; r0 += nt) tiles.push_back(make_int4(p, r0, std::min(nt, n_traj - r0), 0));
}

// Upload tables (pinned staging) and return device pointers.
cr_status upload(Pool& pl, const Tables& t, const ProblemView** px, const ProblemView** pc,
                 const int4** tx, const int4** tc, const int4** sd, const ResultView** rs) {
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o = a256(o + b); return r; };
  const size_t a = take(t.px.size() * sizeof(ProblemView)), b = take(t.pc.size() * sizeof(ProblemView)),
               c = take(t.tx.size() * sizeof(int4)), d = take(t.tc.size() * sizeof(int4)),
               e = take(t.seeds.size() * sizeof(int4)), f = take(t.res.size() * sizeof(ResultView));
  SV_CUDA(cudaStreamSynchronize(pl.stream));  // the previous upload has left the staging buffer
  if (pl.tab_bytes < o) {
    if (pl.tab) cudaFree(pl.tab);
    pl.tab = nullptr;
    pl.tab_bytes = 0;
    SV_CUDA(cudaMalloc(&pl.tab, 2 * o));
    pl.tab_bytes = 2 * o;
  }
  if (pl.tab_host_bytes < o) {
    if (pl.tab_host) cudaFreeHost(pl.tab_host);
    pl.tab_host = nullptr;
    pl.tab_host_bytes = 0;
    SV_CUDA(cudaMallocHost(&pl.tab_host, 2 * o));
    pl.tab_host_bytes = 2 * o;
  }
  unsigned char* h = pl.tab_host;
  if (!t.px.empty()) std::memcpy(h + a, t.px.data(), t.px.size() * sizeof(ProblemView));
  if (!t.pc.empty()) std::memcpy(h + b, t.pc.data(), t.pc.size() * sizeof(ProblemView));
  if (!t.tx.empty()) std::memcpy(h + c, t.tx.data(), t.tx.size() * sizeof(int4));
  if (!t.tc.empty()) std::memcpy(h + d, t.tc.data(), t.tc.size() * sizeof(int4));
  if (!t.seeds.empty()) std::memcpy(h + e, t.seeds.data(), t.seeds.size() * sizeof(int4));
  if (!t.res.empty()) std::memcpy(h + f, t.res.data(), t.res.size() * sizeof(ResultView));
  SV_CUDA(cudaMemcpyAsync(pl.tab, h, o, cudaMemcpyHostToDevice, pl.stream));
  unsigned char* dv = static_cast<unsigned char*>(pl.tab);
  *px = (const ProblemView*)(dv + a);
  *pc = (const ProblemView*)(dv + b);
  *tx = (const int4*)(dv + c);
  *tc = (const int4*)(dv + d);
  *sd = (const int4*)(dv + e);
  *rs = (const ResultView*)(dv + f);
  return CR_OK;
}

cr_status launch_eval_set(cr_server* sv, Pool& pl, const ProblemView* probs, const int4* tiles,
                          int n_tiles, bool cand) {
  if (n_tiles == 0) return CR_OK;
  const cr_opt_state st = pl.state();
  EvalArgs a{};
  std::memset(&a, 0, sizeof(a));
  a.rb = sv->robot->view;
  a.prm = pl.prm;
  a.problems = probs;
  a.tiles = tiles;
  a.n_tiles = n_tiles;
  const int nt = traj_per_tile(pl.H);
  a.max_traj = std::min(nt, cand ? pl.B * pl.na : pl.B);
  a.max_states = a.max_traj * pl.H;
  a.max_horizon = pl.H;
  a.theta = cand ? st.cand : st.x;
  a.cost = cand ? st.cand_cost : st.c;
  a.grad = cand ? st.cand_grad : st.g;
  a.cfree = cand ? st.cand_cfree : st.best_cfree;
  a.no_store_x = -1;
  const int block = kEvalBlock;
  if (eval_smem_bytes(a, block) > eval_smem_limit()) return failf(CR_EINVAL, "server: tile too large");
  const int per_sm = std::max(1, eval_blocks_per_sm(a, block));
  int grid = n_tiles;
  if (n_tiles > per_sm * sv->n_sm) {  // more tiles than resident CTAs: take them from a counter
    a.queue = (int*)pl.p(pl.o_queue);
    grid = per_sm * sv->n_sm;
    SV_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int), pl.stream));
  }
  SV_CUDA(launch_eval(a, grid, block, pl.stream));
  return CR_OK;
}

cr_status launch_opt_set(cr_server* sv, Pool& pl, const int4* seeds, int n_seeds, bool select,
                         bool propose, bool init) {
  if (n_seeds == 0) return CR_OK;
  OptArgs o{};
  std::memset(&o, 0, sizeof(o));
  o.prm = pl.prm;
  o.q_lo = sv->robot->view.lim;
  o.q_hi = sv->robot->view.lim + sv->robot->dof;
  o.dof = sv->robot->dof;
  o.n_seeds = n_seeds;
  o.seed_tab = seeds;
  o.st = pl.state();
  o.do_select = select;
  o.do_propose = propose;
  o.init_best = init;
  SV_CUDA(launch_opt(o, pl.n, pl.stream));
  return CR_OK;
}

// One step of one kind: admit, initialise new requests, iterate, retire.
cr_status step_kind(cr_server* sv, Pool& pl) {
  const int k = pl.kind;
  // 1. admission
  std::vector<int> fresh;
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    Request& r = *sv->reqs[*it];
    if (r.kind != k) {
      ++it;
      continue;
    }
    int cap_limit = sv->cfg.max_active > 0 ? sv->cfg.max_active : (1 << 20);
    int s = free_slot(pl);
    if (s < 0 && pl.capacity < cap_limit) {
      bool grown = false;
      cr_status st = grow(sv, pl, std::min(cap_limit, std::max(4, pl.capacity * 2)), &grown);
      if (st != CR_OK) return st;
      if (grown) s = free_slot(pl);
    }
    if (s < 0) break;  // no memory for another request now: it waits
    r.slot = s;
    pl.slot_req[s] = (int)*it;
    const size_t nv = (size_t)pl.B * pl.n;
    SV_CUDA(cudaMemcpyAsync(pl.p(pl.o_x) + (size_t)s * nv * 4, r.seeds.data(), nv * 4,
                            cudaMemcpyHostToDevice, pl.stream));
    SV_CUDA(cudaMemsetAsync(pl.p(pl.o_s) + (size_t)s * nv * pl.m * 4, 0, nv * pl.m * 4, pl.stream));
    SV_CUDA(cudaMemsetAsync(pl.p(pl.o_y) + (size_t)s * nv * pl.m * 4, 0, nv * pl.m * 4, pl.stream));
    SV_CUDA(cudaMemsetAsync(pl.p(pl.o_rho) + (size_t)s * pl.B * pl.m * 4, 0, (size_t)pl.B * pl.m * 4, pl.stream));
    SV_CUDA(cudaMemsetAsync(pl.p(pl.o_it) + (size_t)s * pl.B * 4, 0, (size_t)pl.B * 4, pl.stream));
    fresh.push_back(s);
    it = sv->queue.erase(it);
  }
  // active slots after admission
  std::vector<int> active;
  for (int s = 0; s < pl.capacity; ++s)
    if (pl.slot_req[s] >= 0) active.push_back(s);
  if (active.empty()) return CR_OK;
  // tables: x-eval for fresh slots, candidate eval + seeds for all active
  Tables t;
  for (size_t q = 0; q < fresh.size(); ++q) {
    ProblemView v;
    cr_status st = slot_view(sv, pl, fresh[q], *sv->reqs[pl.slot_req[fresh[q]]], &v);
    if (st != CR_OK) return st;
    t.px.push_back(v);
    add_tiles(t.tx, (int)q, pl.B, pl.H);
  }
  std::vector<int4> fresh_seeds;
  for (int s : fresh)
    for (int b = 0; b < pl.B; ++b) fresh_seeds.push_back(make_int4(pl.n, (s * pl.B + b) * pl.n, s * pl.B + b, s));
  for (size_t q = 0; q < active.size(); ++q) {
    const int s = active[q];
    ProblemView v;
    cr_status st = slot_view(sv, pl, s, *sv->reqs[pl.slot_req[s]], &v);
    if (st != CR_OK) return st;
    v.n_traj = pl.B * pl.na;
    v.traj_base = s * pl.B * pl.na;
    v.var_base = (long long)s * pl.B * pl.n * pl.na;
    t.pc.push_back(v);
    add_tiles(t.tc, (int)q, pl.B * pl.na, pl.H);
    for (int b = 0; b < pl.B; ++b) t.seeds.push_back(make_int4(pl.n, (s * pl.B + b) * pl.n, s * pl.B + b, s));
  }
  const size_t n_active_seeds = t.seeds.size();
  t.seeds.insert(t.seeds.end(), fresh_seeds.begin(), fresh_seeds.end());
  // result views of the slots that finish in this step
  const int chunk = sv->cfg.chunk;
  std::vector<int> finishing;
  for (int s : active) {
    const Request& r = *sv->reqs[pl.slot_req[s]];
    if (r.iters_done + chunk >= pl.iters) finishing.push_back(s);
  }
  const ResLayout rl(pl.B, pl.n);
  for (size_t q = 0; q < finishing.size(); ++q) {
    const int s = finishing[q];
    unsigned char* r0 = pl.p(pl.o_res) + (size_t)s * rl.bytes;
    ResultView rv;
    rv.traj = (float*)r0;
    rv.cost = (float*)(r0 + rl.cost);
    rv.cfree = (uint8_t*)(r0 + rl.cfree);
    rv.best = (int*)(r0 + rl.best);
    rv.status = nullptr;
    rv.n_seeds = pl.B;
    rv.n = pl.n;
    rv.seed_base = s * pl.B;
    rv.var_base = s * pl.B * pl.n;
    t.res.push_back(rv);
  }
  const ProblemView *px, *pc;
  const int4 *tx, *tc, *sd;
  const ResultView* rs;
  cr_status st = upload(pl, t, &px, &pc, &tx, &tc, &sd, &rs);
  if (st != CR_OK) return st;
  // 2. initial evaluation + first L-BFGS step of the fresh requests
  if (!fresh.empty()) {
    st = launch_eval_set(sv, pl, px, tx, (int)t.tx.size(), false);
    if (st != CR_OK) return st;
    st = launch_opt_set(sv, pl, sd + n_active_seeds, (int)fresh_seeds.size(), false, true, true);
    if (st != CR_OK) return st;
  }
  //    chunk iterations for every active request
  for (int it = 0; it < chunk; ++it) {
    st = launch_eval_set(sv, pl, pc, tc, (int)t.tc.size(), true);
    if (st != CR_OK) return st;
    st = launch_opt_set(sv, pl, sd, (int)n_active_seeds, true, true, false);
    if (st != CR_OK) return st;
  }
  for (int s : active) sv->reqs[pl.slot_req[s]]->iters_done += chunk;
  // 3. retire
  if (!finishing.empty()) {
    SV_CUDA(launch_finish(rs, (int)finishing.size(), (const float*)pl.p(pl.o_bx),
                          (const float*)pl.p(pl.o_bc), (const uint8_t*)pl.p(pl.o_bfree), pl.stream));
  }
  return CR_OK;
}

cr_status collect(cr_server* sv, Pool& pl) {
  const ResLayout rl(pl.B, pl.n);
  for (int s = 0; s < pl.capacity; ++s) {
    if (pl.slot_req[s] < 0) continue;
    Request& r = *sv->reqs[pl.slot_req[s]];
    if (r.iters_done < pl.iters) continue;
    const unsigned char* r0 = pl.p(pl.o_res) + (size_t)s * rl.bytes;
    r.traj.resize((size_t)pl.n * pl.B);
    r.cost.resize(pl.B);
    r.cfree.resize(pl.B);
    int best = -1;
    SV_CUDA(cudaMemcpy(r.traj.data(), r0, r.traj.size() * 4, cudaMemcpyDeviceToHost));
    SV_CUDA(cudaMemcpy(r.cost.data(), r0 + rl.cost, (size_t)pl.B * 4, cudaMemcpyDeviceToHost));
    SV_CUDA(cudaMemcpy(r.cfree.data(), r0 + rl.cfree, pl.B, cudaMemcpyDeviceToHost));
    SV_CUDA(cudaMemcpy(&best, r0 + rl.best, 4, cudaMemcpyDeviceToHost));
    r.best = best;
    r.done = true;
    r.slot = -1;
    pl.slot_req[s] = -1;
  }
  return CR_OK;
}

}  // namespace

extern "C" {

cr_status cr_server_create(cr_ctx* ctx, const cr_robot* robot, const cr_server_config* cfg,
                           cr_server** out) {
  if (!ctx || !robot || !cfg || !out) return failf(CR_EINVAL, "cr_server_create: null argument");
  *out = nullptr;
  if (cfg->chunk < 1) return failf(CR_EINVAL, "cr_server_create: chunk < 1");
  std::unique_ptr<cr_server> sv(new cr_server());
  sv->ctx = ctx;
  sv->robot = robot;
  sv->cfg = *cfg;
  int dev = 0;
  SV_CUDA(cudaGetDevice(&dev));
  SV_CUDA(cudaDeviceGetAttribute(&sv->n_sm, cudaDevAttrMultiProcessorCount, dev));
  for (int k = 0; k < 2; ++k) {
    Pool& pl = sv->pool[k];
    cr_status st = check_params(&cfg->kind_params[k]);
    if (st != CR_OK) return st;
    pl.kind = k;
    pl.B = cfg->kind_seeds[k];
    pl.H = cfg->kind_horizon[k];
    pl.iters = cfg->kind_iters[k];
    if (pl.B < 1 || pl.H < 1 || pl.H > kMaxHorizon || pl.iters < 1)
      return failf(CR_EINVAL, "cr_server_create: kind %d: bad seeds / horizon / iterations", k);
    if (pl.iters % cfg->chunk != 0)
      return failf(CR_EINVAL, "cr_server_create: kind %d: iterations must be a multiple of chunk", k);
    pl.n = pl.H * robot->dof;
    if (pl.n > 2048) return failf(CR_EINVAL, "cr_server_create: horizon * dof > 2048");
    pl.prm = cfg->kind_params[k];
    pl.m = pl.prm.history;
    pl.na = pl.prm.n_alpha;
    SV_CUDA(cudaStreamCreateWithFlags(&pl.stream, cudaStreamNonBlocking));
  }
  *out = sv.release();
  return CR_OK;
}

void cr_server_destroy(cr_server* sv) { delete sv; }

cr_status cr_server_submit(cr_server* sv, int32_t kind, const cr_problem* pr, uint64_t* ticket) {
  if (!sv || !pr || !ticket || kind < 0 || kind > 1) return failf(CR_EINVAL, "cr_server_submit: bad argument");
  const Pool& pl = sv->pool[kind];
  if (!pr->world || !pr->q_start || !pr->goal || !pr->seeds)
    return failf(CR_EINVAL, "cr_server_submit: null field");
  if (pr->n_seeds != pl.B || pr->horizon != pl.H)
    return failf(CR_EINVAL, "cr_server_submit: kind %d takes %d seeds x %d steps", kind, pl.B, pl.H);
  std::unique_ptr<Request> r(new Request());
  r->ticket = sv->next_ticket++;
  r->kind = kind;
  r->world = pr->world;
  const int D = sv->robot->dof;
  r->q_start.assign(pr->q_start, pr->q_start + D);
  r->goal.assign(pr->goal, pr->goal + 7);
  r->seeds.assign(pr->seeds, pr->seeds + (size_t)pl.B * pl.n);
  *ticket = r->ticket;
  sv->by_ticket[r->ticket] = sv->reqs.size();
  sv->queue.push_back(sv->reqs.size());
  sv->reqs.push_back(std::move(r));
  return CR_OK;
}

cr_status cr_server_step(cr_server* sv, void* stream) {
  if (!sv) return failf(CR_EINVAL, "cr_server_step: null server");
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t ev;
  SV_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  SV_CUDA(cudaEventRecord(ev, cs));
  for (auto& pl : sv->pool) SV_CUDA(cudaStreamWaitEvent(pl.stream, ev, 0));
  // both kinds enqueue on their own streams, so their kernels overlap
  for (auto& pl : sv->pool) {
    cr_status st = step_kind(sv, pl);
    if (st != CR_OK) {
      cudaEventDestroy(ev);
      return st;
    }
  }
  for (auto& pl : sv->pool) SV_CUDA(cudaStreamSynchronize(pl.stream));
  cudaEventDestroy(ev);
  for (auto& pl : sv->pool) {
    cr_status st = collect(sv, pl);
    if (st != CR_OK) return st;
  }
  return CR_OK;
}

cr_status cr_server_poll(cr_server* sv, uint64_t ticket, int32_t* done, float* traj, float* cost,
                         uint8_t* cfree, int32_t* best) {
  if (!sv || !done) return failf(CR_EINVAL, "cr_server_poll: null argument");
  auto it = sv->by_ticket.find(ticket);
  if (it == sv->by_ticket.end()) return failf(CR_EINVAL, "cr_server_poll: unknown ticket");
  Request& r = *sv->reqs[it->second];
  *done = r.done ? 1 : 0;
  if (!r.done) return CR_OK;
  if (traj) std::memcpy(traj, r.traj.data(), r.traj.size() * 4);
  if (cost) std::memcpy(cost, r.cost.data(), r.cost.size() * 4);
  if (cfree) std::memcpy(cfree, r.cfree.data(), r.cfree.size());
  if (best) *best = r.best;
  return CR_OK;
}

cr_status cr_server_stats(cr_server* sv, int32_t* active, int32_t* queued, size_t* pool_bytes) {
  if (!sv) return failf(CR_EINVAL, "cr_server_stats: null server");
  int a = 0;
  size_t b = 0;
  for (auto& pl : sv->pool) {
    for (int s = 0; s < pl.capacity; ++s) a += pl.slot_req[s] >= 0;
    b += pl.bytes;
  }
  if (active) *active = a;
  if (queued) *queued = (int32_t)sv->queue.size();
  if (pool_bytes) *pool_bytes = b;
  return CR_OK;
}

}  // extern "C"
