// k_particle.cu -- particle-based optimisation (Sec. 4.2, Eq. 12-13,
// Alg. "Particle-Based Optimization"): SAMPLE and UPDATE kernels and the
// cr_particle_step entry point (the cost of the particles is the fused
// evaluation kernel, without gradients).
#include <cuda_runtime.h>

#include <cstdio>

#include "crgb_internal.cuh"

namespace crgb {

namespace {

// particles[b][i][k] = mu[b][k] + sqrt(sigma[b][k]) * eps[b][i][k]
__global__ void k_particle_sample(const float* __restrict__ mu, const float* __restrict__ sigma,
                                  const float* __restrict__ eps, float* __restrict__ particles,
                                  int n, int n_p, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / ((long long)n_p * n);
    const int k = (int)(e % n);
    const long long v = b * n + k;
    particles[e] = fmaf(sqrtf(sigma[v]), eps[e], mu[v]);
  }
}

// UPDATE of one seed on one CTA: exponential utility of c = -cost / beta,
// taken after subtracting the smallest cost (w unchanged); every thread forms
// the same normaliser in particle order.  Then per variable, in particle
// order: Eq. 12 mean and Eq. 13 covariance (weighted second moment about the
// previous mean).  c [n_p] costs, th [n_p][n] particles, mu / sigma [n].
__device__ __forceinline__ void particle_update_seed(const float* c, const float* th, float* mu, float* sigma,
                                                     int n, int n_p, float inv_beta, float k_mu, float k_sigma,
                                                     float* s_w) {
  float cmin = c[0];
  for (int i = 1; i < n_p; ++i) cmin = fminf(cmin, c[i]);
  for (int i = threadIdx.x; i < n_p; i += blockDim.x) s_w[i] = expf(-(c[i] - cmin) * inv_beta);
  __syncthreads();
  float z = 0.f;
  for (int i = 0; i < n_p; ++i) z += s_w[i];
  const float inv_z = 1.f / z;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float m0 = mu[k];
    float m = 0.f, s2 = 0.f;
    for (int i = 0; i < n_p; ++i) {
      const float w = s_w[i] * inv_z;
      const float t = th[(long long)i * n + k];
      m = fmaf(w, t, m);
      const float d = t - m0;
      s2 = fmaf(w, d * d, s2);
    }
    sigma[k] = fmaf(1.f - k_sigma, sigma[k], k_sigma * s2);
    mu[k] = fmaf(1.f - k_mu, m0, k_mu * m);
  }
}

// One CTA per seed of one problem.
__global__ void k_particle_update(const float* __restrict__ cost, const float* __restrict__ particles,
                                  float* __restrict__ mu, float* __restrict__ sigma, int n, int n_p,
                                  float inv_beta, float k_mu, float k_sigma) {
  extern __shared__ float s_w[];  // [n_p]
  const int b = blockIdx.x;
  particle_update_seed(cost + (long long)b * n_p, particles + (long long)b * n_p * n, mu + (long long)b * n,
                       sigma + (long long)b * n, n, n_p, inv_beta, k_mu, k_sigma, s_w);
}

// The seeds of a batch of uneven problems (seed table rows: n variables,
// variable offset, seed index, problem): particles and samples of seed s at
// n_p x its variable offset, its costs at n_p x its index.
__global__ void k_particle_sample_tab(const int4* __restrict__ seed_tab, const float* __restrict__ mu,
                                      const float* __restrict__ sigma, const float* __restrict__ eps,
                                      float* __restrict__ particles, int n_p) {
  const int4 e = seed_tab[blockIdx.x];
  const int n = e.x;
  const long long vo = e.y;
  for (int q = threadIdx.x; q < n_p * n; q += blockDim.x) {
    const int k = q % n;
    const long long at = vo * n_p + q;
    particles[at] = fmaf(sqrtf(sigma[vo + k]), eps[at], mu[vo + k]);
  }
}

__global__ void k_particle_update_tab(const int4* __restrict__ seed_tab, const float* __restrict__ cost,
                                      const float* __restrict__ particles, float* __restrict__ mu,
                                      float* __restrict__ sigma, int n_p, float inv_beta, float k_mu,
                                      float k_sigma) {
  extern __shared__ float s_w[];  // [n_p]
  const int4 e = seed_tab[blockIdx.x];
  const long long vo = e.y;
  particle_update_seed(cost + (long long)e.z * n_p, particles + vo * n_p, mu + vo, sigma + vo, e.x, n_p,
                       inv_beta, k_mu, k_sigma, s_w);
}

__global__ void k_fill(float* __restrict__ p, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

cudaError_t launch_particle_batch(const int4* seed_tab, int n_seeds, int n_p, int phase, const float* eps,
                                  float* mu, float* sigma, float* particles, const float* cost, float beta,
                                  float k_mu, float k_sigma, cudaStream_t s) {
  if (n_seeds <= 0) return cudaSuccess;
  if (phase == 0)
    k_particle_sample_tab<<<n_seeds, 256, 0, s>>>(seed_tab, mu, sigma, eps, particles, n_p);
  else
    k_particle_update_tab<<<n_seeds, 256, (size_t)n_p * sizeof(float), s>>>(seed_tab, cost, particles, mu, sigma,
                                                                            n_p, 1.f / beta, k_mu, k_sigma);
  return cudaGetLastError();
}

cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  k_fill<<<(int)(want < 152 * 8 ? want : 152 * 8), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace crgb

using namespace crgb;

extern "C" cr_status cr_particle_step(const cr_robot* robot, const cr_problem* problem,
                                      const cr_params* params, int32_t n_seeds, int32_t n_particles,
                                      float* mu, float* sigma, const float* eps, float* particles,
                                      float* cost, float beta, float k_mu, float k_sigma,
                                      void* stream) {
  if (!robot || !problem) return set_error(CR_EINVAL, "cr_particle_step: null robot or problem");
  if (n_seeds < 0 || n_particles < 1 || n_particles > 4096)
    return set_error(CR_EINVAL, "cr_particle_step: n_seeds < 0 or n_particles outside 1..4096");
  if (!(beta > 0.f) || !(k_mu >= 0.f && k_mu <= 1.f) || !(k_sigma >= 0.f && k_sigma <= 1.f))
    return set_error(CR_EINVAL, "cr_particle_step: beta must be > 0, k_mu and k_sigma in [0, 1]");
  if (n_seeds == 0) return CR_OK;
  if (!mu || !sigma || !eps || !particles || !cost)
    return set_error(CR_EINVAL, "cr_particle_step: null buffer");
  const int n = problem->horizon * robot->dof;
  const long long total = (long long)n_seeds * n_particles * n;
  if ((long long)n_seeds * n_particles > 0x7fffffffLL)
    return set_error(CR_EINVAL, "cr_particle_step: too many particles");
  cudaStream_t s = (cudaStream_t)stream;
  const int blk = 256;
  const long long want = (total + blk - 1) / blk;
  const int grid = (int)(want < 152 * 16 ? want : 152 * 16);
  k_particle_sample<<<grid, blk, 0, s>>>(mu, sigma, eps, particles, n, n_particles, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  cr_status st = cr_eval(robot, problem, params, particles, n_seeds * n_particles, cost, nullptr,
                         nullptr, nullptr, nullptr, stream);
  if (st != CR_OK) return st;
  k_particle_update<<<n_seeds, 256, (size_t)n_particles * sizeof(float), s>>>(
      cost, particles, mu, sigma, n, n_particles, 1.f / beta, k_mu, k_sigma);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  return CR_OK;
}
