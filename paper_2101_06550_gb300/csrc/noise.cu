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
#include "noise.cuh"

using namespace chx;

namespace {

constexpr int kThreads = 256;

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
    float x0, y0, x1, y1;
    deviate_pair(b, step, seed, sim0 + (uint64_t)z, &x0, &y0, &x1, &y1);
    rx[2 * b] = x0;
    ry[2 * b] = y0;
    if (2 * b + 1 < np) {
      rx[2 * b + 1] = x1;
      ry[2 * b + 1] = y1;
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
