// server.cu -- continuous batching of motion-generation and IK requests
// with device-resident optimiser state and admission by free device memory.
//
// Requests of two kinds (0: trajectory optimisation / motion generation,
// 1: IK) carry their own seed count and horizon; the kind fixes the
// parameters and the iteration count.  Requests of one kind and one shape
// (seeds, horizon) share a pool: every per-seed array of the optimiser
// (iterate, gradient, history, candidates, best iterate) is one device array
// with room for `capacity` slots, slot s owning seeds s*B .. s*B + B - 1.
// Each pool has its own stream and runs independently of the others.
//
// cr_server_step does not wait for the device, except while a pool grows or
// its table buffer is enlarged (the live slots are copied over and the old
// arrays freed, which can wait for the device).  For every pool it
//   1. collects the pool's last round if the round has finished (results of
//      the requests that retired in it, already copied to pinned host
//      memory; their slots become free);
//   2. admits queued requests into free slots of idle pools, growing a pool
//      (doubling, the live slots copied over) only while free device memory
//      minus the reserve allows;
//   3. starts a round on every idle pool with active requests: the initial
//      evaluation and first L-BFGS step of the new ones, then `chunk`
//      iterations for all (one evaluation launch over the line-search
//      candidates of every active request, one selection + L-BFGS launch over
//      their seeds), then the results of the requests that reach their
//      iteration count, copied to pinned host memory; an event marks the end.
// So a request that arrives while a pool is busy is admitted as soon as that
// pool's round ends, and pools of other shapes or kinds keep running.
// A request's arithmetic never depends on the other requests, so its result
// is bit-identical to cr_solve of that request alone; a request's optimiser
// state can be copied out (cr_server_snapshot) and continued in another
// server (cr_server_restore) with the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
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

constexpr int kMaxPools = 64;

// Result staging of one slot: traj [B][n] | cost [B] | cfree [B] | best | status.
struct ResLayout {
  size_t cost, cfree, best, status, bytes;
  ResLayout(int B, int n) {
    cost = (size_t)B * n * 4;
    cfree = cost + (size_t)B * 4;
    best = (cfree + B + 3) & ~size_t(3);
    status = best + 4;
    bytes = a256(status + 4);
  }
};

int traj_per_tile(int H) { return H >= 32 ? 1 : (32 + H - 1) / H; }

struct Request {
  uint64_t ticket = 0;
  int kind = 0, B = 0, H = 0;
  const cr_world* world = nullptr;
  std::vector<float> q_start, goal, goal_q, seeds;
  std::vector<unsigned char> restored;  // optimiser state of a restored request (snapshot layout)
  int pool = -1, slot = -1;
  int iters_done = 0;
  bool done = false;
  std::vector<float> traj, cost;
  std::vector<uint8_t> cfree;
  int best = -1, status = CR_OK;
};

// Field-major device pool of one request shape.
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
  // per-round tables (device and pinned staging)
  void* tab = nullptr;
  size_t tab_bytes = 0;
  unsigned char* tab_host = nullptr;
  size_t tab_host_bytes = 0;
  // results of the slots retiring in the running round, pinned
  unsigned char* res_host = nullptr;
  size_t res_host_bytes = 0;
  std::vector<int> retiring;  // slots whose results the running round copies out
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  bool busy = false;

  ~Pool() {
    if (base) cudaFree(base);
    if (tab) cudaFree(tab);
    if (tab_host) cudaFreeHost(tab_host);
    if (res_host) cudaFreeHost(res_host);
    if (done_ev) cudaEventDestroy(done_ev);
    if (stream) cudaStreamDestroy(stream);
  }

  // carve-up for `cap` slots; returns total bytes
  size_t layout(int cap, size_t* f) const {
    const size_t S = (size_t)cap * B, V = S * n;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o = a256(o + b); return r; };
    f[0] = take(V * 4); f[1] = take(V * 4); f[2] = take(V * 4); f[3] = take(V * 4);
    f[4] = take(V * 4); f[5] = take(V * 4); f[6] = take(S * 4); f[7] = take(S * 4);
    f[8] = take(S * m * 4); f[9] = take(S * 4); f[10] = take(V * m * 4); f[11] = take(V * m * 4);
    f[12] = take(V * na * 4); f[13] = take(V * na * 4); f[14] = take(S * na * 4);
    f[15] = take(S * na); f[16] = take(S); f[17] = take(S * 4); f[18] = take(256);
    f[19] = take((size_t)cap * ResLayout(B, n).bytes);  // result staging
    return o;
  }
  void set_offsets(const size_t* f) {
    o_x = f[0]; o_g = f[1]; o_xp = f[2]; o_gp = f[3]; o_dir = f[4]; o_bx = f[5]; o_c = f[6]; o_bc = f[7];
    o_rho = f[8]; o_it = f[9]; o_s = f[10]; o_y = f[11]; o_cand = f[12]; o_cgrad = f[13]; o_ccost = f[14];
    o_cfree = f[15]; o_bfree = f[16]; o_ls = f[17]; o_queue = f[18]; o_res = f[19];
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

// The optimiser state of one request (one slot) as a snapshot stores it:
// every field the next iteration reads (the candidates' costs, gradients and
// flags are recomputed by it).
struct StateField {
  size_t Pool::*off;
  bool per_var;  // elements per seed: n (per variable) or 1
  int elem;      // bytes per element
  int mult;      // 0: x1, 1: x m (history), 2: x n_alpha (candidates)
};
const StateField kStateFields[] = {
    {&Pool::o_x, true, 4, 0},    {&Pool::o_g, true, 4, 0},   {&Pool::o_c, false, 4, 0},
    {&Pool::o_xp, true, 4, 0},   {&Pool::o_gp, true, 4, 0},  {&Pool::o_s, true, 4, 1},
    {&Pool::o_y, true, 4, 1},    {&Pool::o_rho, false, 4, 1}, {&Pool::o_it, false, 4, 0},
    {&Pool::o_dir, true, 4, 0},  {&Pool::o_cand, true, 4, 2}, {&Pool::o_bx, true, 4, 0},
    {&Pool::o_bc, false, 4, 0},  {&Pool::o_bfree, false, 1, 0}, {&Pool::o_ls, false, 4, 0},
};

// bytes one slot holds of a field
size_t field_bytes(const Pool& pl, const StateField& f) {
  size_t e = (size_t)pl.B * (f.per_var ? (size_t)pl.n : 1) * f.elem;
  if (f.mult == 1) e *= pl.m;
  if (f.mult == 2) e *= pl.na;
  return e;
}

size_t state_bytes(const Pool& pl) {
  size_t t = 0;
  for (const StateField& f : kStateFields) t += field_bytes(pl, f);
  return t;
}

}  // namespace

struct cr_server {
  cr_ctx* ctx = nullptr;
  const cr_robot* robot = nullptr;
  cr_server_config cfg{};
  std::vector<std::unique_ptr<Pool>> pools;
  std::vector<std::unique_ptr<Request>> reqs;  // every submitted request
  std::map<uint64_t, size_t> by_ticket;
  std::deque<size_t> queue;                    // waiting for a slot
  uint64_t next_ticket = 1;
  int n_sm = 0;
  cudaEvent_t ev_in = nullptr;
  ~cr_server() {
    for (auto& pl : pools)
      if (pl->stream) cudaStreamSynchronize(pl->stream);
    pools.clear();
    if (ev_in) cudaEventDestroy(ev_in);
  }
};

namespace {

int find_pool(cr_server* sv, int kind, int B, int H) {
  for (size_t i = 0; i < sv->pools.size(); ++i) {
    const Pool& p = *sv->pools[i];
    if (p.kind == kind && p.B == B && p.H == H) return (int)i;
  }
  return -1;
}

cr_status make_pool(cr_server* sv, int kind, int B, int H, int* out) {
  if ((int)sv->pools.size() >= kMaxPools)
    return failf(CR_EINVAL, "server: more than %d request shapes", kMaxPools);
  std::unique_ptr<Pool> pl(new Pool());
  pl->kind = kind;
  pl->B = B;
  pl->H = H;
  pl->n = H * sv->robot->dof;
  pl->iters = sv->cfg.kind_iters[kind];
  pl->prm = sv->cfg.kind_params[kind];
  pl->m = pl->prm.history;
  pl->na = pl->prm.n_alpha;
  SV_CUDA(cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking));
  SV_CUDA(cudaEventCreateWithFlags(&pl->done_ev, cudaEventDisableTiming));
  sv->pools.push_back(std::move(pl));
  *out = (int)sv->pools.size() - 1;
  return CR_OK;
}

// Grow an idle pool to `cap` slots when free memory minus the reserve allows,
// copying the live slots' state (field by field) into the new arrays.
cr_status grow(cr_server* sv, Pool& pl, int cap, bool* grown) {
  *grown = false;
  size_t f[20];
  const size_t need = pl.layout(cap, f);
  size_t free_b = 0, total_b = 0;
  SV_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t extra = need > pl.bytes ? need - pl.bytes : 0;
  if (free_b < sv->cfg.reserve_bytes || free_b - sv->cfg.reserve_bytes < extra) return CR_OK;
  void* nb = nullptr;
  if (cudaMalloc(&nb, need) != cudaSuccess) {
    cudaGetLastError();
    return CR_OK;  // refused: requests keep waiting
  }
  const size_t res_need = (size_t)cap * ResLayout(pl.B, pl.n).bytes;
  if (pl.res_host_bytes < res_need) {
    if (pl.res_host) cudaFreeHost(pl.res_host);
    pl.res_host = nullptr;
    pl.res_host_bytes = 0;
    if (cudaMallocHost(&pl.res_host, res_need) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(nb);
      return CR_OK;
    }
    pl.res_host_bytes = res_need;
  }
  if (pl.base) {
    SV_CUDA(cudaStreamSynchronize(pl.stream));
    size_t old[20];
    pl.layout(pl.capacity, old);
    const size_t S0 = (size_t)pl.capacity * pl.B, V0 = S0 * pl.n;
    const size_t sizes[18] = {V0 * 4, V0 * 4, V0 * 4, V0 * 4, V0 * 4, V0 * 4, S0 * 4, S0 * 4,
                              S0 * pl.m * 4, S0 * 4, V0 * pl.m * 4, V0 * pl.m * 4, V0 * pl.na * 4,
                              V0 * pl.na * 4, S0 * pl.na * 4, S0 * pl.na, S0, S0 * 4};
    for (int k = 0; k < 18; ++k)
      SV_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(nb) + f[k], pl.p(old[k]), sizes[k],
                              cudaMemcpyDeviceToDevice, pl.stream));
    SV_CUDA(cudaStreamSynchronize(pl.stream));
    cudaFree(pl.base);
  }
  pl.base = nb;
  pl.bytes = need;
  pl.capacity = cap;
  pl.set_offsets(f);
  pl.slot_req.resize(cap, -1);
  *grown = true;
  return CR_OK;
}

int free_slot(const Pool& pl) {
  for (int s = 0; s < pl.capacity; ++s)
    if (pl.slot_req[s] < 0) return s;
  return -1;
}

// Tables of one round for a pool: problem views for the iterate (x) or
// candidate evaluation, tiles, seed table, result views.
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
  pr.goal_q = r.goal_q.empty() ? nullptr : r.goal_q.data();
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

// Upload tables (pinned staging; the pool is idle, so the previous round's
// upload has left the buffer) and return device pointers.
cr_status upload(Pool& pl, const Tables& t, const ProblemView** px, const ProblemView** pc,
                 const int4** tx, const int4** tc, const int4** sd, const ResultView** rs) {
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o = a256(o + b); return r; };
  const size_t a = take(t.px.size() * sizeof(ProblemView)), b = take(t.pc.size() * sizeof(ProblemView)),
               c = take(t.tx.size() * sizeof(int4)), d = take(t.tc.size() * sizeof(int4)),
               e = take(t.seeds.size() * sizeof(int4)), f = take(t.res.size() * sizeof(ResultView));
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

// The results of the round that just finished: requests that retired in it.
void collect(cr_server* sv, Pool& pl) {
  const ResLayout rl(pl.B, pl.n);
  for (int s : pl.retiring) {
    const int ri = pl.slot_req[s];
    if (ri < 0) continue;
    Request& r = *sv->reqs[ri];
    const unsigned char* r0 = pl.res_host + (size_t)s * rl.bytes;
    r.traj.assign((const float*)r0, (const float*)r0 + (size_t)pl.B * pl.n);
    r.cost.assign((const float*)(r0 + rl.cost), (const float*)(r0 + rl.cost) + pl.B);
    r.cfree.assign(r0 + rl.cfree, r0 + rl.cfree + pl.B);
    std::memcpy(&r.best, r0 + rl.best, 4);
    std::memcpy(&r.status, r0 + rl.status, 4);
    r.done = true;
    r.slot = -1;
    r.pool = -1;
    pl.slot_req[s] = -1;
  }
  pl.retiring.clear();
  pl.busy = false;
}

// Collect every pool whose round has ended.
cr_status poll_pools(cr_server* sv) {
  for (auto& up : sv->pools) {
    Pool& pl = *up;
    if (!pl.busy) continue;
    cudaError_t e = cudaEventQuery(pl.done_ev);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) return failf(CR_ECUDA, "server round: %s", cudaGetErrorString(e));
    collect(sv, pl);
  }
  return CR_OK;
}

// Put a request into a free slot of its (idle) pool: its seeds with an empty
// history, or the state of a restored request.  *fresh = it needs its
// initial evaluation and first step.
cr_status admit(cr_server* sv, Pool& pl, size_t ri, int s, bool* fresh) {
  Request& r = *sv->reqs[ri];
  r.slot = s;
  pl.slot_req[s] = (int)ri;
  const size_t nv = (size_t)pl.B * pl.n;
  if (!r.restored.empty()) {
    const unsigned char* src = r.restored.data();
    for (const StateField& f : kStateFields) {
      const size_t fb = field_bytes(pl, f);
      SV_CUDA(cudaMemcpyAsync(pl.p(pl.*(f.off)) + (size_t)s * fb, src, fb, cudaMemcpyHostToDevice, pl.stream));
      src += fb;
    }
    *fresh = false;
    return CR_OK;
  }
  SV_CUDA(cudaMemcpyAsync(pl.p(pl.o_x) + (size_t)s * nv * 4, r.seeds.data(), nv * 4, cudaMemcpyHostToDevice,
                          pl.stream));
  SV_CUDA(cudaMemsetAsync(pl.p(pl.o_s) + (size_t)s * nv * pl.m * 4, 0, nv * pl.m * 4, pl.stream));
  SV_CUDA(cudaMemsetAsync(pl.p(pl.o_y) + (size_t)s * nv * pl.m * 4, 0, nv * pl.m * 4, pl.stream));
  SV_CUDA(cudaMemsetAsync(pl.p(pl.o_rho) + (size_t)s * pl.B * pl.m * 4, 0, (size_t)pl.B * pl.m * 4, pl.stream));
  SV_CUDA(cudaMemsetAsync(pl.p(pl.o_it) + (size_t)s * pl.B * 4, 0, (size_t)pl.B * 4, pl.stream));
  *fresh = true;
  return CR_OK;
}

// One round of an idle pool: initialise the fresh requests, run `chunk`
// iterations for every active one, copy out those that finish.
cr_status start_round(cr_server* sv, Pool& pl, const std::vector<int>& fresh) {
  std::vector<int> active;
  for (int s = 0; s < pl.capacity; ++s)
    if (pl.slot_req[s] >= 0) active.push_back(s);
  if (active.empty()) return CR_OK;
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
  const int chunk = sv->cfg.chunk;
  pl.retiring.clear();
  for (int s : active) {
    const Request& r = *sv->reqs[pl.slot_req[s]];
    if (r.iters_done + chunk >= pl.iters) pl.retiring.push_back(s);
  }
  const ResLayout rl(pl.B, pl.n);
  for (int s : pl.retiring) {
    unsigned char* r0 = pl.p(pl.o_res) + (size_t)s * rl.bytes;
    ResultView rv;
    rv.traj = (float*)r0;
    rv.cost = (float*)(r0 + rl.cost);
    rv.cfree = (uint8_t*)(r0 + rl.cfree);
    rv.best = (int*)(r0 + rl.best);
    rv.status = (int*)(r0 + rl.status);
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
  if (!fresh.empty()) {
    st = launch_eval_set(sv, pl, px, tx, (int)t.tx.size(), false);
    if (st != CR_OK) return st;
    st = launch_opt_set(sv, pl, sd + n_active_seeds, (int)fresh_seeds.size(), false, true, true);
    if (st != CR_OK) return st;
  }
  for (int it = 0; it < chunk; ++it) {
    st = launch_eval_set(sv, pl, pc, tc, (int)t.tc.size(), true);
    if (st != CR_OK) return st;
    st = launch_opt_set(sv, pl, sd, (int)n_active_seeds, true, true, false);
    if (st != CR_OK) return st;
  }
  for (int s : active) sv->reqs[pl.slot_req[s]]->iters_done += chunk;
  if (!pl.retiring.empty()) {
    SV_CUDA(launch_finish(rs, (int)pl.retiring.size(), (const float*)pl.p(pl.o_bx), (const float*)pl.p(pl.o_bc),
                          (const uint8_t*)pl.p(pl.o_bfree), pl.stream));
    for (int s : pl.retiring)
      SV_CUDA(cudaMemcpyAsync(pl.res_host + (size_t)s * rl.bytes, pl.p(pl.o_res) + (size_t)s * rl.bytes, rl.bytes,
                              cudaMemcpyDeviceToHost, pl.stream));
  }
  SV_CUDA(cudaEventRecord(pl.done_ev, pl.stream));
  pl.busy = true;
  return CR_OK;
}

// ---- snapshot layout: header | q_start | goal | goal_q | seeds | state ----
constexpr uint32_t kSnapMagic = 0x56535243u;  // "CRSV"
constexpr uint32_t kSnapVersion = 1;

struct SnapHeader {
  uint32_t magic, version;
  int32_t kind, B, H, dof, m, na, iters_done, has_state, has_goal_q, pad;
  cr_params prm;
};

size_t snap_bytes(int B, int H, int dof, bool goal_q, size_t state) {
  return sizeof(SnapHeader) + 4 * ((size_t)dof + 7 + (goal_q ? dof : 0) + (size_t)B * H * dof) + state;
}

cr_status queue_request(cr_server* sv, std::unique_ptr<Request> r, uint64_t* ticket) {
  if (sv->cfg.max_queued > 0 && (int)sv->queue.size() >= sv->cfg.max_queued)
    return failf(CR_EBUSY, "server: %d requests already wait for a slot", (int)sv->queue.size());
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->by_ticket[r->ticket] = sv->reqs.size();
  sv->queue.push_back(sv->reqs.size());
  sv->reqs.push_back(std::move(r));
  return CR_OK;
}

}  // namespace

extern "C" {

cr_status cr_server_create(cr_ctx* ctx, const cr_robot* robot, const cr_server_config* cfg,
                           cr_server** out) {
  if (!ctx || !robot || !cfg || !out) return failf(CR_EINVAL, "cr_server_create: null argument");
  *out = nullptr;
  if (cfg->chunk < 1) return failf(CR_EINVAL, "cr_server_create: chunk < 1");
  if (cfg->max_queued < 0 || cfg->max_active < 0) return failf(CR_EINVAL, "cr_server_create: negative limit");
  for (int k = 0; k < 2; ++k) {
    cr_status st = check_params(&cfg->kind_params[k]);
    if (st != CR_OK) return st;
    if (cfg->kind_iters[k] < 1) return failf(CR_EINVAL, "cr_server_create: kind %d: iterations < 1", k);
    if (cfg->kind_iters[k] % cfg->chunk != 0)
      return failf(CR_EINVAL, "cr_server_create: kind %d: iterations must be a multiple of chunk", k);
  }
  if (!(cfg->kind_params[1].flags & CR_IK_MODE))
    return failf(CR_EINVAL, "cr_server_create: kind 1 (IK) needs CR_IK_MODE");
  std::unique_ptr<cr_server> sv(new cr_server());
  sv->ctx = ctx;
  sv->robot = robot;
  sv->cfg = *cfg;
  int dev = 0;
  SV_CUDA(cudaGetDevice(&dev));
  SV_CUDA(cudaDeviceGetAttribute(&sv->n_sm, cudaDevAttrMultiProcessorCount, dev));
  SV_CUDA(cudaEventCreateWithFlags(&sv->ev_in, cudaEventDisableTiming));
  *out = sv.release();
  return CR_OK;
}

void cr_server_destroy(cr_server* sv) { delete sv; }

cr_status cr_server_submit(cr_server* sv, int32_t kind, const cr_problem* pr, uint64_t* ticket) {
  if (!sv || !pr || !ticket || kind < 0 || kind > 1) return failf(CR_EINVAL, "cr_server_submit: bad argument");
  if (!pr->world || !pr->q_start || !pr->goal || !pr->seeds)
    return failf(CR_EINVAL, "cr_server_submit: null field");
  const int B = pr->n_seeds, H = pr->horizon, D = sv->robot->dof;
  if (B < 1 || H < 1 || H > kMaxHorizon) return failf(CR_EINVAL, "cr_server_submit: bad seed count or horizon");
  if (H * D > 2048) return failf(CR_EINVAL, "cr_server_submit: horizon * dof > 2048");
  if (kind == 1 && H != 1) return failf(CR_EINVAL, "cr_server_submit: IK requests (kind 1) take horizon 1");
  std::unique_ptr<Request> r(new Request());
  r->kind = kind;
  r->B = B;
  r->H = H;
  r->world = pr->world;
  r->q_start.assign(pr->q_start, pr->q_start + D);
  r->goal.assign(pr->goal, pr->goal + 7);
  if (pr->goal_q) r->goal_q.assign(pr->goal_q, pr->goal_q + D);
  r->seeds.assign(pr->seeds, pr->seeds + (size_t)B * H * D);
  return queue_request(sv, std::move(r), ticket);
}

cr_status cr_server_step(cr_server* sv, void* stream) {
  if (!sv) return failf(CR_EINVAL, "cr_server_step: null server");
  // 1. rounds that have ended
  cr_status st = poll_pools(sv);
  if (st != CR_OK) return st;
  // work of this step follows the caller's stream
  SV_CUDA(cudaEventRecord(sv->ev_in, (cudaStream_t)stream));
  // 2. admission into idle pools, first come first served per pool
  std::vector<std::vector<int>> fresh(sv->pools.size());
  std::vector<char> full(sv->pools.size(), 0), waited(sv->pools.size(), 0);
  const int cap_limit = sv->cfg.max_active > 0 ? sv->cfg.max_active : (1 << 20);
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    Request& r = *sv->reqs[*it];
    int pi = find_pool(sv, r.kind, r.B, r.H);
    if (pi < 0) {
      st = make_pool(sv, r.kind, r.B, r.H, &pi);
      if (st != CR_OK) return st;
      fresh.resize(sv->pools.size());
      full.resize(sv->pools.size(), 0);
      waited.resize(sv->pools.size(), 0);
    }
    Pool& pl = *sv->pools[pi];
    if (pl.busy || full[pi]) {
      ++it;
      continue;
    }
    int s = free_slot(pl);
    if (s < 0 && pl.capacity < cap_limit) {
      bool grown = false;
      st = grow(sv, pl, std::min(cap_limit, std::max(4, pl.capacity * 2)), &grown);
      if (st != CR_OK) return st;
      if (grown) s = free_slot(pl);
    }
    if (s < 0) {  // no slot and no memory for one now: it and later requests of this pool wait
      full[pi] = 1;
      ++it;
      continue;
    }
    if (!waited[pi]) {
      SV_CUDA(cudaStreamWaitEvent(pl.stream, sv->ev_in, 0));
      waited[pi] = 1;
    }
    bool is_fresh = false;
    st = admit(sv, pl, *it, s, &is_fresh);
    if (st != CR_OK) return st;
    r.pool = pi;
    if (is_fresh) fresh[pi].push_back(s);
    it = sv->queue.erase(it);
  }
  // 3. a round on every idle pool with active requests
  for (size_t pi = 0; pi < sv->pools.size(); ++pi) {
    Pool& pl = *sv->pools[pi];
    if (pl.busy || pl.capacity == 0) continue;
    if (!waited[pi]) SV_CUDA(cudaStreamWaitEvent(pl.stream, sv->ev_in, 0));
    st = start_round(sv, pl, fresh[pi]);
    if (st != CR_OK) return st;
  }
  return CR_OK;
}

cr_status cr_server_poll(cr_server* sv, uint64_t ticket, int32_t* done, float* traj, float* cost,
                         uint8_t* cfree, int32_t* best, int32_t* status) {
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
  if (status) *status = r.status;
  return CR_OK;
}

cr_status cr_server_wait(cr_server* sv, uint64_t ticket, int32_t timeout_ms) {
  if (!sv) return failf(CR_EINVAL, "cr_server_wait: null server");
  auto it = sv->by_ticket.find(ticket);
  if (it == sv->by_ticket.end()) return failf(CR_EINVAL, "cr_server_wait: unknown ticket");
  const size_t ri = it->second;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cr_status st = cr_server_step(sv, nullptr);
    if (st != CR_OK) return st;
    if (sv->reqs[ri]->done) return CR_OK;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0 && ms >= timeout_ms)
      return failf(CR_ETIMEOUT, "cr_server_wait: request %llu not finished after %d ms",
                   (unsigned long long)ticket, timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

cr_status cr_server_snapshot(cr_server* sv, uint64_t ticket, void* buf, size_t* bytes) {
  if (!sv || !bytes) return failf(CR_EINVAL, "cr_server_snapshot: null argument");
  auto it = sv->by_ticket.find(ticket);
  if (it == sv->by_ticket.end()) return failf(CR_EINVAL, "cr_server_snapshot: unknown ticket");
  Request& r = *sv->reqs[it->second];
  // a request in a running round: wait for the round (it may retire)
  if (r.pool >= 0 && sv->pools[r.pool]->busy) {
    Pool& pl = *sv->pools[r.pool];
    SV_CUDA(cudaEventSynchronize(pl.done_ev));
    collect(sv, pl);
  }
  if (r.done) return failf(CR_EINVAL, "cr_server_snapshot: request %llu has finished", (unsigned long long)ticket);
  const int D = sv->robot->dof;
  const bool admitted = r.slot >= 0;
  const size_t state = admitted ? state_bytes(*sv->pools[r.pool]) : r.restored.size();
  const size_t need = snap_bytes(r.B, r.H, D, !r.goal_q.empty(), state);
  if (!buf) {
    *bytes = need;
    return CR_OK;
  }
  if (*bytes < need) {
    const size_t have = *bytes;
    *bytes = need;
    return failf(CR_EINVAL, "cr_server_snapshot: buffer of %zu bytes, %zu needed", have, need);
  }
  *bytes = need;
  SnapHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  hd.magic = kSnapMagic;
  hd.version = kSnapVersion;
  hd.kind = r.kind;
  hd.B = r.B;
  hd.H = r.H;
  hd.dof = D;
  hd.m = sv->cfg.kind_params[r.kind].history;
  hd.na = sv->cfg.kind_params[r.kind].n_alpha;
  hd.iters_done = r.iters_done;
  hd.has_state = state > 0;
  hd.has_goal_q = !r.goal_q.empty();
  hd.prm = sv->cfg.kind_params[r.kind];
  unsigned char* o = static_cast<unsigned char*>(buf);
  std::memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  auto put = [&](const std::vector<float>& v) {
    if (!v.empty()) std::memcpy(o, v.data(), v.size() * 4);
    o += v.size() * 4;
  };
  put(r.q_start);
  put(r.goal);
  put(r.goal_q);
  put(r.seeds);
  if (admitted) {
    Pool& pl = *sv->pools[r.pool];
    for (const StateField& f : kStateFields) {
      const size_t fb = field_bytes(pl, f);
      SV_CUDA(cudaMemcpyAsync(o, pl.p(pl.*(f.off)) + (size_t)r.slot * fb, fb, cudaMemcpyDeviceToHost, pl.stream));
      o += fb;
    }
    SV_CUDA(cudaStreamSynchronize(pl.stream));
  } else if (!r.restored.empty()) {
    std::memcpy(o, r.restored.data(), r.restored.size());
  }
  return CR_OK;
}

cr_status cr_server_restore(cr_server* sv, const void* buf, size_t bytes, const cr_world* world,
                            uint64_t* ticket) {
  if (!sv || !buf || !world || !ticket) return failf(CR_EINVAL, "cr_server_restore: null argument");
  SnapHeader hd;
  if (bytes < sizeof(hd)) return failf(CR_EINVAL, "cr_server_restore: buffer too small");
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kSnapMagic || hd.version != kSnapVersion)
    return failf(CR_EINVAL, "cr_server_restore: not a request snapshot of this library");
  const int D = sv->robot->dof;
  if (hd.kind < 0 || hd.kind > 1 || hd.dof != D || hd.B < 1 || hd.H < 1 || hd.H > kMaxHorizon)
    return failf(CR_EINVAL, "cr_server_restore: snapshot of another robot or shape");
  if (std::memcmp(&hd.prm, &sv->cfg.kind_params[hd.kind], sizeof(cr_params)) != 0)
    return failf(CR_EINVAL, "cr_server_restore: the server's parameters for this kind differ from the snapshot's");
  if (hd.iters_done < 0 || hd.iters_done >= sv->cfg.kind_iters[hd.kind] || hd.iters_done % sv->cfg.chunk != 0)
    return failf(CR_EINVAL, "cr_server_restore: iteration count %d does not fit this server", hd.iters_done);
  Pool probe;
  probe.B = hd.B;
  probe.n = hd.H * D;
  probe.m = hd.m;
  probe.na = hd.na;
  const size_t state = hd.has_state ? state_bytes(probe) : 0;
  if (bytes != snap_bytes(hd.B, hd.H, D, hd.has_goal_q != 0, state))
    return failf(CR_EINVAL, "cr_server_restore: snapshot size does not match its header");
  std::unique_ptr<Request> r(new Request());
  r->kind = hd.kind;
  r->B = hd.B;
  r->H = hd.H;
  r->world = world;
  r->iters_done = hd.iters_done;
  const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof(hd);
  auto get = [&](std::vector<float>& v, size_t count) {
    v.resize(count);
    if (count) std::memcpy(v.data(), p, count * 4);
    p += count * 4;
  };
  get(r->q_start, D);
  get(r->goal, 7);
  get(r->goal_q, hd.has_goal_q ? D : 0);
  get(r->seeds, (size_t)hd.B * hd.H * D);
  if (hd.has_state) r->restored.assign(p, p + state);
  return queue_request(sv, std::move(r), ticket);
}

cr_status cr_server_stats(cr_server* sv, int32_t* active, int32_t* queued, size_t* pool_bytes) {
  if (!sv) return failf(CR_EINVAL, "cr_server_stats: null server");
  int a = 0;
  size_t b = 0;
  for (auto& pl : sv->pools) {
    for (int s = 0; s < pl->capacity; ++s) a += pl->slot_req[s] >= 0;
    b += pl->bytes;
  }
  if (active) *active = a;
  if (queued) *queued = (int32_t)sv->queue.size();
  if (pool_bytes) *pool_bytes = b;
  return CR_OK;
}

}  // extern "C"
