// k_retime.cu -- retiming of App. "Time-step Discretization" (Alg. "Time
// Discretization"): the time step that puts a trajectory at the robot's
// velocity, acceleration or jerk limit.  The App. A.5 stencils scale as
// 1/dt, 1/dt^2, 1/dt^3, so from the stencils at dt = 1 the smallest dt that
// keeps every sample within the limits is the largest of |v1|/v_max,
// sqrt(|a1|/a_max), cbrt(|j1|/j_max).
#include <cuda_runtime.h>

#include "crgb_internal.cuh"
#include "k_time.cuh"

namespace crgb {

namespace {

// One warp per trajectory; a maximum, so the order of the samples is free.
__global__ void k_retime(RobotView rb, ProblemView pv, const float* __restrict__ theta, int B,
                         float* __restrict__ dt_out) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= B) return;
  const int D = rb.dof, H = pv.horizon;
  float dt = retime_part(theta + (long long)b * H * D, pv.q_start, rb.lim, H, D, lane, 32);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dt = fmaxf(dt, __shfl_xor_sync(0xffffffffu, dt, o));
  if (lane == 0) dt_out[b] = dt;
}

}  // namespace

}  // namespace crgb

using namespace crgb;

extern "C" cr_status cr_retime(const cr_robot* robot, const cr_problem* problem, int32_t B,
                               const float* theta, float* dt, void* stream) {
  if (!robot || !problem) return set_error(CR_EINVAL, "cr_retime: null robot or problem");
  if (B < 0) return set_error(CR_EINVAL, "cr_retime: B < 0");
  if (B == 0) return CR_OK;
  if (!theta || !dt) return set_error(CR_EINVAL, "cr_retime: null buffer");
  ProblemView pv;
  cr_status st = fill_problem(robot, problem, &pv, nullptr);
  if (st != CR_OK) return st;
  const int warps = 8;
  k_retime<<<(B + warps - 1) / warps, 32 * warps, 0, (cudaStream_t)stream>>>(robot->view, pv, theta, B, dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  return CR_OK;
}
