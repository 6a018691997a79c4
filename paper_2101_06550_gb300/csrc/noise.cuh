// Device generator of the Cahn-Hilliard-Cook deviates (Sec. 7.7), shared by the
// standalone deviate kernel and the right-hand-side pass that draws them in
// place.  Counter-based Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011):
// points 2b and 2b + 1 of step t of simulation `sim` take the four words of
// Philox(counter = (b, t, 0, 0), key = (seed, sim)).  Word w gives
// u = (floor(w / 2^41) + 1/2) 2^-23, exact in FP32 and inside (0, 1); the pairs
// (u0, u1) and (u2, u3) give (rho^x, rho^y) of the two points as
// sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub), evaluated in FP32.
#pragma once
#include <stdint.h>

namespace chx {

__device__ __forceinline__ void philox4x64_10(uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t& x3, uint64_t k0,
                                              uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
    const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
    const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
  }
}

__device__ __forceinline__ float unit_open(uint64_t w) { return ((float)(w >> 41) + 0.5f) * 0x1p-23f; }

__device__ __forceinline__ void box_muller(uint64_t wa, uint64_t wb, float* zx, float* zy) {
  const float rad = sqrtf(-2.0f * logf(unit_open(wa)));
  float s, c;
  sincospif(2.0f * unit_open(wb), &s, &c);
  *zx = rad * c;
  *zy = rad * s;
}

// The deviates of the pair b = (points 2b, 2b + 1) of step `step`, key (seed, sim).
__device__ __forceinline__ void deviate_pair(uint64_t b, uint64_t step, uint64_t seed, uint64_t sim, float* x0,
                                             float* y0, float* x1, float* y1) {
  uint64_t w0 = b, w1 = step, w2 = 0, w3 = 0;
  philox4x64_10(w0, w1, w2, w3, seed, sim);
  box_muller(w0, w1, x0, y0);
  box_muller(w2, w3, x1, y1);
}

}  // namespace chx
