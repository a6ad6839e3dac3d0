// k_steer.cu -- parallel steering (Sec. 5, Alg. "Parallel Steering"): edges
// discretised into n + 1 samples, every sample checked by the fused
// evaluation's discrete clearance test (mask_samples), and per edge the last
// valid sample before the first invalid one.
#include <cuda_runtime.h>

#include <cmath>

#include "crgb_internal.cuh"

namespace crgb {

namespace {

// samples[e][i] = a_e + (i / n)(b_e - a_e), i = 0..n
__global__ void k_steer_samples(const float* __restrict__ edges, int E, int n, int D,
                                float* __restrict__ samples) {
  const long long total = (long long)E * (n + 1) * D;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k % D);
    const long long ei = k / D;
    const int i = (int)(ei % (n + 1));
    const long long e = ei / (n + 1);
    const float a = edges[(e * 2) * D + j], b = edges[(e * 2 + 1) * D + j];
    samples[k] = fmaf((float)i / (float)n, b - a, a);
  }
}

// one thread per edge: first invalid sample, last valid one, its distance
__global__ void k_steer_reduce(const float* __restrict__ edges, const uint8_t* __restrict__ ok, int E,
                               int n, int D, int32_t* __restrict__ last, float* __restrict__ v_new,
                               float* __restrict__ dist) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int h = n;
  for (int i = 0; i <= n; ++i)
    if (!ok[(long long)e * (n + 1) + i]) {
      h = i - 1;
      break;
    }
  last[e] = h;
  const float s = h < 0 ? 0.f : (float)h / (float)n;
  float d2 = 0.f;
  for (int j = 0; j < D; ++j) {
    const float a = edges[((long long)e * 2) * D + j], b = edges[((long long)e * 2 + 1) * D + j];
    const float v = fmaf(s, b - a, a);
    v_new[(long long)e * D + j] = v;
    d2 = fmaf(v - a, v - a, d2);
  }
  dist[e] = sqrtf(d2);
}

}  // namespace

}  // namespace crgb

using namespace crgb;

extern "C" cr_status cr_steer(const cr_robot* robot, const cr_world* world, int32_t n_edges,
                              const float* edges, int32_t n, float* samples, uint8_t* valid,
                              float* cost, int32_t* last, float* v_new, float* dist, void* stream) {
  if (!robot || !world) return set_error(CR_EINVAL, "cr_steer: null robot or world");
  if (n_edges < 0 || n < 1) return set_error(CR_EINVAL, "cr_steer: n_edges < 0 or n < 1");
  if (n_edges == 0) return CR_OK;
  if (!edges || !samples || !valid || !cost || !last || !v_new || !dist)
    return set_error(CR_EINVAL, "cr_steer: null buffer");
  if ((long long)n_edges * (n + 1) > 0x7fffffffLL) return set_error(CR_EINVAL, "cr_steer: too many samples");
  const int D = robot->dof;
  cudaStream_t s = (cudaStream_t)stream;
  const long long total = (long long)n_edges * (n + 1) * D;
  const long long want = (total + 255) / 256;
  k_steer_samples<<<(int)(want < 152 * 16 ? want : 152 * 16), 256, 0, s>>>(edges, n_edges, n, D, samples);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  // every sample as a single-state problem: the evaluation's discrete test
  // (every sphere clear of every box, every pair of S separated)
  cr_params prm;
  cr_params_default(&prm);
  prm.flags = CR_IK_MODE | CR_SELF;
  float q0[CR_MAX_DOF] = {0.f};
  const float goal[7] = {0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f};
  cr_problem pr = {};
  pr.world = world;
  pr.q_start = q0;
  pr.goal = goal;
  pr.horizon = 1;
  cr_status st = cr_eval(robot, &pr, &prm, samples, n_edges * (n + 1), cost, nullptr, valid, nullptr, nullptr, stream);
  if (st != CR_OK) return st;
  k_steer_reduce<<<(n_edges + 127) / 128, 128, 0, s>>>(edges, valid, n_edges, n, D, last, v_new, dist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  return CR_OK;
}
