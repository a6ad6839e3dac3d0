// fastdiv.h -- quotient of a non-negative int by a divisor that stays the same
// over many divisions (a tile's horizon, the robot's sphere or joint count),
// with one high multiply, an add and a shift instead of a full integer
// division.  This is the method of Granlund and Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994, Sec. 4): for a divisor
// d >= 1 let l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, which is
// below 2^32; then for 0 <= n < 2^31
//     n / d = (hi32(m n) + n) >> l,
// and the sum stays below 2^32 because hi32(m n) <= n.  Plain C++ on the
// host, so the same header is checked exhaustively against '/' by a CPU test.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define CR_FD_HD __host__ __device__ __forceinline__
#else
#define CR_FD_HD inline
#endif

namespace crgb {

struct FastDiv {
  uint32_t m;  // multiplier
  uint32_t l;  // shift, ceil(log2 d)
  int32_t d;   // divisor (for remainders)
};

// d < 1 is taken as 1 (a loop over zero items never divides)
CR_FD_HD FastDiv make_fastdiv(int32_t d) {
  FastDiv f;
  if (d < 1) d = 1;
  uint32_t l = 0;
  while ((1ull << l) < (uint64_t)d) ++l;
  f.l = l;
  f.m = (uint32_t)(((((uint64_t)1 << l) - (uint64_t)d) << 32) / (uint64_t)d + 1ull);
  f.d = d;
  return f;
}

CR_FD_HD uint32_t fd_hi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// n / d for 0 <= n < 2^31
CR_FD_HD int32_t fdiv(int32_t n, const FastDiv& f) {
  return (int32_t)((fd_hi32((uint32_t)n, f.m) + (uint32_t)n) >> f.l);
}

}  // namespace crgb
