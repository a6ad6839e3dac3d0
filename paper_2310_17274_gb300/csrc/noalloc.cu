// noalloc.cu -- batched evaluation of several problems in one persistent
// launch, for callers that cannot allocate device memory.
//
// The regular batched path keeps its tile and problem tables and its work
// counter in a workspace it allocates (and grows) on demand.  Some callers
// cannot let a library allocate: a robot controller's real-time loop that
// must not call cudaMalloc/cudaFree once it runs (those calls can take
// unbounded time and synchronise the device), or a host application that
// hands every byte of device memory to its own pool and forbids libraries
// from allocating behind its back.  This entry point serves them: its scratch
// (tables + counter) lives in one file-scope device array of fixed size that
// every GPU loading the library holds until the process exits; the caller
// passes inputs and outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "crgb_internal.cuh"

using namespace crgb;

namespace crgb {
cr_status check_params(const cr_params* p);
}  // namespace crgb

namespace {

constexpr int kNoAllocProblems = CR_NOALLOC_MAX_PROBLEMS;
constexpr int kNoAllocTiles = CR_NOALLOC_MAX_TILES;
constexpr size_t kProbBytes = sizeof(ProblemView) * kNoAllocProblems;
constexpr size_t kTileOff = (kProbBytes + 255) & ~size_t(255);
constexpr size_t kTileBytes = sizeof(int4) * kNoAllocTiles;
constexpr size_t kQueueOff = (kTileOff + kTileBytes + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kQueueOff + 256;

// problem table | tile table | work counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// device address of the scratch array per device, looked up once; host
// threads making their first call on a device at the same time each store the
// same address
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices] = {};

cr_status fail(cr_status code, const char* msg) { return set_error(code, msg); }

int traj_per_tile(int H) { return H >= 32 ? 1 : (32 + H - 1) / H; }

}  // namespace

extern "C" cr_status cr_eval_batch_noalloc(const cr_robot* robot, int32_t n_problems,
                                           const cr_problem* problems, const cr_params* params,
                                           const int32_t* n_traj, const float* theta, float* cost,
                                           float* grad, uint8_t* cfree, float* terms, void* stream) {
  if (!robot || !problems || !n_traj) return fail(CR_EINVAL, "cr_eval_batch_noalloc: null argument");
  if (n_problems < 1 || n_problems > kNoAllocProblems)
    return fail(CR_EINVAL, "cr_eval_batch_noalloc: n_problems outside 1..CR_NOALLOC_MAX_PROBLEMS (256)");
  cr_status s = check_params(params);
  if (s != CR_OK) return s;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CR_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CR_EINVAL, "cr_eval_batch_noalloc: device index >= 64");
  cudaStream_t st = (cudaStream_t)stream;
  {
    // the tables below are copied from host memory that lives only during
    // this call: a captured copy would read it after it is gone
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return fail(CR_ECUDA, cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(CR_EINVAL, "cr_eval_batch_noalloc: the stream is being captured (the call stages its "
                             "tables from temporary host memory and cannot be recorded)");
  }
  unsigned char* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(CR_ECUDA, cudaGetErrorString(e));
    scratch = static_cast<unsigned char*>(p);
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }

  std::vector<ProblemView> pv(n_problems);
  std::vector<int4> tiles;
  long long vo = 0;
  int tb = 0, max_traj = 0, max_states = 0, max_h = 0;
  for (int p = 0; p < n_problems; ++p) {
    s = fill_problem(robot, &problems[p], &pv[p], params);
    if (s != CR_OK) return s;
    if (n_traj[p] < 0) return fail(CR_EINVAL, "cr_eval_batch_noalloc: n_traj < 0");
    const int H = problems[p].horizon;
    pv[p].n_traj = n_traj[p];
    pv[p].traj_base = tb;
    pv[p].var_base = vo;
    const int nt = traj_per_tile(H);
    for (int r0 = 0; r0 < n_traj[p]; r0 += nt) {
      const int c = std::min(nt, n_traj[p] - r0);
      if ((int)tiles.size() >= kNoAllocTiles)
        return fail(CR_EINVAL, "cr_eval_batch_noalloc: more than CR_NOALLOC_MAX_TILES (32768) tiles");
      tiles.push_back(make_int4(p, r0, c, 0));
      max_traj = std::max(max_traj, c);
      max_states = std::max(max_states, c * H);
    }
    max_h = std::max(max_h, H);
    vo += (long long)n_traj[p] * H * robot->dof;
    tb += n_traj[p];
  }
  if (tiles.empty()) return CR_OK;
  if (!theta || !cost) return fail(CR_EINVAL, "cr_eval_batch_noalloc: null theta or cost");

  e = cudaMemcpyAsync(scratch, pv.data(), pv.size() * sizeof(ProblemView), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scratch + kTileOff, tiles.data(), tiles.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
  // the counter keeps the last call's value: it must start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kQueueOff, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(CR_ECUDA, cudaGetErrorString(e));

  EvalArgs a{};
  std::memset(&a, 0, sizeof(a));
  a.rb = robot->view;
  a.prm = *params;
  a.problems = reinterpret_cast<const ProblemView*>(scratch);
  a.tiles = reinterpret_cast<const int4*>(scratch + kTileOff);
  a.n_tiles = (int)tiles.size();
  a.queue = reinterpret_cast<int*>(scratch + kQueueOff);
  a.max_traj = max_traj;
  a.max_states = max_states;
  a.max_horizon = max_h;
  a.theta = theta;
  a.cost = cost;
  a.grad = grad;
  a.cfree = cfree;
  a.terms = terms;
  a.no_store_x = -1;
  const int block = kEvalBlock;
  if (eval_smem_bytes(a, block) > eval_smem_limit())
    return fail(CR_EINVAL, "cr_eval_batch_noalloc: a tile needs more than 227 KB of shared memory");
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = std::max(1, eval_blocks_per_sm(a, block));
  const int grid = std::min(a.n_tiles, per_sm * n_sm);
  e = launch_eval(a, grid, block, st);
  if (e != cudaSuccess) return fail(CR_ECUDA, cudaGetErrorString(e));
  return CR_OK;
}
