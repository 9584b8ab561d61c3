// Register-ring helpers of the boxcar bank, shared by the search kernels
// (boxcar.cu) and the logsumexp kernels (lse.cu).
//
// A lane owns kR = 33 consecutive start bins k0..k0+32 and keeps their
// running sums s_i = S_w[k0+i] in registers.  Step w adds P[k0+i+w-1] to s_i
// (the recursion of §2.2.5 applied per bin).  The 33 window values live in a
// register ring b, which takes one new shared-memory load per step; with the
// width loop unrolled by 33 every ring index is a compile-time constant.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace ps {

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Fast mode: steps C0 .. C0+NC-1 of the 33-step ring, adds only.
template <int C0, int NC>
__device__ __forceinline__ void fast_steps(float (&s)[kR], float (&b)[kR], const float *__restrict__ pb) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    const int c = C0 + cc;
    b[(c + kR - 1) % kR] = pb[c + kR - 1];
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += b[(i + c) % kR];
  }
}

// Reload the ring after an exact run that ended at step CE of the block:
// the ring must hold positions [33 bi + CE, 33 bi + CE + 31].
template <int CE>
__device__ __forceinline__ void reload_ring(float (&b)[kR], const float *__restrict__ pb) {
#pragma unroll
  for (int j = 0; j < kR - 1; ++j) b[(CE + j) % kR] = pb[CE + j];
}

// Plain steps w = wa..wb-1 (no ring, no compares): the partial last block.
__device__ __forceinline__ void tail_steps(float (&s)[kR], const float *__restrict__ lane_buf, int wa, int wb) {
  for (int w = wa; w < wb; ++w) {
    const float *pw = lane_buf + (w - 1);
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += pw[i];
  }
}

}  // namespace ps
