// Allocation-free variant of the mass / free-energy reduction (ch_diagnostics).
//
// The reduction needs scratch for one partial sum triple per grid row.  Here
// that scratch is a file-scope __device__ array instead of plan-owned device
// memory, so the entry point performs no allocation at all, not even a plan:
// it is meant for callers that must not call cudaMalloc (for example code that
// runs where the allocator is off limits, or a host that has reserved all
// device memory up front).  The array holds kStaticRows rows (384 KiB of
// doubles); every GPU that loads this library keeps it until the process exits.
#include <mutex>

#include "chx_internal.cuh"

using namespace chx;

namespace {

constexpr int kStaticRows = 16384;
constexpr int kRowThreads = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_row_partials[3 * kStaticRows];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One block per row j: mass, energy and a non-finite count of that row.
__global__ void __launch_bounds__(kRowThreads) diag_row_kernel(const double* __restrict__ c, int nx, int ny, double hx,
                                                               double hy, double* __restrict__ part) {
  const int j = blockIdx.x;
  const double* row = c + (size_t)j * nx;
  const double* up = c + (size_t)(j + 1 == ny ? 0 : j + 1) * nx;
  double sm = 0.0, se = 0.0, bad = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = row[i];
    const double gx = row[i + 1 == nx ? 0 : i + 1] - v, gy = up[i] - v;
    const double q = fma(v, v, -1.0);
    sm += v;
    se += 0.25 * q * q + hx * gx * gx + hy * gy * gy;
    if (!isfinite(v)) bad += 1.0;
  }
  __shared__ double s[3][kRowThreads / 32];
  sm = warp_sum(sm);
  se = warp_sum(se);
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0) {
    s[0][threadIdx.x >> 5] = sm;
    s[1][threadIdx.x >> 5] = se;
    s[2][threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0;
    for (int w = 0; w < kRowThreads / 32; ++w) { a += s[0][w]; b += s[1][w]; d += s[2][w]; }
    part[3 * (size_t)j] = a;
    part[3 * (size_t)j + 1] = b;
    part[3 * (size_t)j + 2] = d;
  }
}

// Sums the row partials in row order; a non-finite input makes both results NaN.
__global__ void diag_row_final_kernel(const double* __restrict__ part, int ny, double cell, double* mass,
                                      double* energy) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0, b = 0, d = 0;
  for (int j = 0; j < ny; ++j) { a += part[3 * j]; b += part[3 * j + 1]; d += part[3 * j + 2]; }
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  *mass = d != 0.0 ? nan : a * cell;
  *energy = d != 0.0 ? nan : b * cell;
}

// Device address of the static scratch for the current device, looked up once
// per device (host code cannot use the symbol's host-side stand-in).
int scratch_address(double** out) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "ch_diagnostics_noalloc: cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return fail(CHX_EUNSUPPORTED, "ch_diagnostics_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_row_partials), "ch_diagnostics_noalloc: cudaGetSymbolAddress");
    if (rc) return rc;
    g_addr[dev] = p;
  }
  *out = (double*)g_addr[dev];
  return CHX_OK;
}

}  // namespace

extern "C" int ch_diagnostics_noalloc(const double* c, int nx, int ny, double lx, double ly, double gamma,
                                      double* mass_out, double* energy_out, void* stream) {
  if (!c || !mass_out || !energy_out) return fail(CHX_EINVAL, "ch_diagnostics_noalloc: null pointer");
  if (nx < 1 || ny < 1) return fail(CHX_EINVAL, "ch_diagnostics_noalloc: nx %d, ny %d", nx, ny);
  if (ny > kStaticRows)
    return fail(CHX_EINVAL, "ch_diagnostics_noalloc: ny = %d exceeds the static scratch limit of %d rows", ny,
                kStaticRows);
  if (!(lx > 0) || !(ly > 0) || !(gamma >= 0))
    return fail(CHX_EINVAL, "ch_diagnostics_noalloc: lx %g, ly %g, gamma %g", lx, ly, gamma);
  double* part = nullptr;
  int rc = scratch_address(&part);
  if (rc) return rc;
  const double dx = lx / nx, dy = ly / ny;
  cudaStream_t st = (cudaStream_t)stream;
  diag_row_kernel<<<ny, kRowThreads, 0, st>>>(c, nx, ny, 0.5 * gamma / (dx * dx), 0.5 * gamma / (dy * dy), part);
  diag_row_final_kernel<<<1, 32, 0, st>>>(part, ny, dx * dy, mass_out, energy_out);
  return launch_check("ch_diagnostics_noalloc");
}
