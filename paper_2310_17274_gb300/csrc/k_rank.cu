// k_rank.cu -- choosing among the seeds a solve returns (App. "Solver
// details"): IK returns the valid seed with the lowest weighted sum of pose
// error and distance from the current configuration; trajectory optimisation
// the valid seed with the lowest blend of pose error, largest jerk and motion
// time.  One thread scores a seed; one CTA then takes the lowest score among
// the collision-free seeds (the lowest index on ties, an order-free rule).
#include <cuda_runtime.h>
#include <math.h>

#include "crgb_internal.cuh"
#include "k_device.cuh"
#include "k_time.cuh"

namespace crgb {

namespace {

__global__ void k_rank_score(RobotView rb, ProblemView pv, const float* __restrict__ theta, int B,
                             const float* __restrict__ dt, float dt_all, int ik, RankWeights w,
                             float* __restrict__ score) {
  __shared__ float s_fix[(kMaxDof + 1) * 12];
  __shared__ int s_axis[kMaxDof];
  const int D = rb.dof, H = pv.horizon;
  for (int k = threadIdx.x; k < (D + 1) * 12; k += blockDim.x) s_fix[k] = rb.fixed_tf[k];
  for (int k = threadIdx.x; k < D; k += blockDim.x) s_axis[k] = rb.axis[k];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  score[b] = seed_score(s_fix, s_axis, D, pv, theta + (long long)b * H * D, dt ? dt[b] : dt_all, ik, w);
}

// The lowest score among collision-free seeds, the lowest index on ties; -1
// when there is none.  Scores that are NaN never win.
__global__ void k_rank_best(const float* __restrict__ score, const uint8_t* __restrict__ cfree, int B,
                            int* __restrict__ best) {
  __shared__ float s_s[32];
  __shared__ int s_i[32];
  float bs = INFINITY;
  int bi = -1;
  auto better = [](float s, int i, float bs, int bi) { return score_better(s, i, bs, bi); };
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float s = score[b];
    if (cfree[b] && better(s, b, bs, bi)) {
      bs = s;
      bi = b;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, bs, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi >= 0 && better(os, oi, bs, bi)) {
      bs = os;
      bi = oi;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    s_s[warp] = bs;
    s_i[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w)
      if (s_i[w] >= 0 && better(s_s[w], s_i[w], bs, bi)) {
        bs = s_s[w];
        bi = s_i[w];
      }
    *best = bi;
  }
}

}  // namespace

}  // namespace crgb

using namespace crgb;

extern "C" cr_status cr_rank_seeds(const cr_robot* robot, const cr_problem* problem, const cr_params* params,
                                   int32_t B, const float* theta, const uint8_t* cfree, const float* dt,
                                   float w_pose, float w_jerk, float w_time, float w_dist, float* score,
                                   int32_t* best, void* stream) {
  if (!robot || !problem || !params) return set_error(CR_EINVAL, "cr_rank_seeds: null robot, problem or params");
  if (B < 0) return set_error(CR_EINVAL, "cr_rank_seeds: B < 0");
  if (!score || !best || (B > 0 && (!theta || !cfree)))
    return set_error(CR_EINVAL, "cr_rank_seeds: null buffer");
  const int ik = (params->flags & CR_IK_MODE) != 0;
  if (!ik && !dt && !(params->dt > 0.f)) return set_error(CR_EINVAL, "cr_rank_seeds: dt must be > 0");
  ProblemView pv;
  cr_status st = fill_problem(robot, problem, &pv, params);
  if (st != CR_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  if (B > 0) {
    const RankWeights w{w_pose, w_jerk, w_time, w_dist};
    k_rank_score<<<(B + 127) / 128, 128, 0, s>>>(robot->view, pv, theta, B, dt, params->dt, ik, w, score);
  }
  k_rank_best<<<1, 256, 0, s>>>(score, cfree, B, best);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  return CR_OK;
}
