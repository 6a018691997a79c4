// Normal deviates for the Cahn-Hilliard-Cook forcing (Sec. 7.7): a 2-vector
// field rho of N(0, 1) numbers per grid point, drawn afresh every step by the
// Box-Muller transform of uniforms.
//
// The uniforms come from the counter-based generator Philox4x64-10 (Salmon,
// Moraes, Dror, Shaw, SC 2011), so any point of any step is computed
// independently: points 2b and 2b + 1 of step t of simulation `sim` take the
// four words of Philox(counter = (b, t, 0, 0), key = (seed, sim)).  Word w
// gives u = (floor(w / 2^41) + 1/2) 2^-23, exact in FP32 and inside (0, 1);
// the pairs (u0, u1) and (u2, u3) give (rho^x, rho^y) of the two points as
// sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub).  The transform is evaluated in
// FP32 (the deviates only scale a forcing of intensity sqrt(sigma)); the values
// are stored as FP64 for the FP64 right-hand side.
#include <stdint.h>

#include "chx_internal.cuh"

using namespace chx;

namespace {

constexpr int kThreads = 256;

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

__device__ __forceinline__ void box_muller(uint64_t wa, uint64_t wb, double* zx, double* zy) {
  const float rad = sqrtf(-2.0f * logf(unit_open(wa)));
  float s, c;
  sincospif(2.0f * unit_open(wb), &s, &c);
  *zx = (double)(rad * c);
  *zy = (double)(rad * s);
}

// rho: G fields of [rho^x (nx*ny), rho^y (nx*ny)]; field z uses key (seed, sim0 + z).
// The step index is `step`, or *d_step when d_step is given (a device counter
// that captured graphs advance with step_advance_kernel).
__global__ void __launch_bounds__(kThreads) noise_normals_kernel(double* __restrict__ rho, size_t np, uint64_t seed,
                                                                 uint64_t sim0, uint64_t step,
                                                                 const uint64_t* __restrict__ d_step) {
  if (d_step) step = *d_step;
  const size_t pairs = (np + 1) / 2;
  const int z = blockIdx.y;
  double* rx = rho + (size_t)z * 2 * np;
  double* ry = rx + np;
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < pairs; b += (size_t)gridDim.x * blockDim.x) {
    uint64_t x0 = b, x1 = step, x2 = 0, x3 = 0;
    philox4x64_10(x0, x1, x2, x3, seed, sim0 + (uint64_t)z);
    double zx, zy;
    box_muller(x0, x1, &zx, &zy);
    rx[2 * b] = zx;
    ry[2 * b] = zy;
    if (2 * b + 1 < np) {
      box_muller(x2, x3, &zx, &zy);
      rx[2 * b + 1] = zx;
      ry[2 * b + 1] = zy;
    }
  }
}

__global__ void step_advance_kernel(uint64_t* d_step) { *d_step += 1; }
__global__ void step_set_kernel(uint64_t* d_step, uint64_t v) { *d_step = v; }

}  // namespace

namespace chx {
int launch_step_set(uint64_t* d_step, uint64_t v, cudaStream_t st) {
  step_set_kernel<<<1, 1, 0, st>>>(d_step, v);
  return launch_check("noise step counter");
}

int launch_step_advance(uint64_t* d_step, cudaStream_t st) {
  step_advance_kernel<<<1, 1, 0, st>>>(d_step);
  return launch_check("noise step counter");
}

int launch_noise_normals(double* rho, int nx, int ny, int G, uint64_t seed, uint64_t sim0, uint64_t step,
                         const uint64_t* d_step, cudaStream_t st) {
  const size_t np = (size_t)nx * ny, pairs = (np + 1) / 2;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = ceil_div(pairs, (size_t)kThreads), cap = (size_t)sms * 8;
  const dim3 grid((unsigned)(want < cap ? want : cap), (unsigned)G);
  noise_normals_kernel<<<grid, kThreads, 0, st>>>(rho, np, seed, sim0, step, d_step);
  return launch_check("noise_normals");
}
}  // namespace chx

extern "C" int ch_noise_normals(double* rho, int nx, int ny, uint64_t seed, uint64_t sim, uint64_t step, void* stream) {
  if (!rho || nx < 1 || ny < 1) return fail(CHX_EINVAL, "ch_noise_normals: rho %p, nx %d, ny %d", (void*)rho, nx, ny);
  return launch_noise_normals(rho, nx, ny, 1, seed, sim, step, nullptr, (cudaStream_t)stream);
}
