// Coarsening observables of Cahn-Hilliard fields (Secs. 2.4, 3.5.4, 7.2.3):
//   mass = sum C dx dy,
//   F_h  = sum [ (1/4)(C^2 - 1)^2 + (gamma/2)(|D+x C|^2 + |D+y C|^2) ] dx dy,
//   s    = 1 / (1 - <C^2>), <.> the composite Simpson average (periodic closure:
//          weights (2, 4, 2, 4, ...)/3 per direction for an even count, the
//          trapezoid rule for an odd one),
//   k1   = sum |C^(k)|^2 / sum |k|^-1 |C^(k)|^2 over the Fourier modes k != 0.
// One launch covers every slot of a group (blockIdx.y); sums run in a fixed
// order, so results are bit-reproducible.  The Fourier transform for k1 is a
// plain library FFT (cuFFT, real-to-complex); the weighted spectral sums are
// this file's kernels.
#include <cufft.h>
#include <math.h>

#include "chgroup.cuh"

namespace chx {

struct ObsState {
  double* part = nullptr;
  size_t part_cap = 0;  // doubles
  cufftHandle fft = 0;
  bool fft_ok = false;
  int fft_batch = 0;        // fields the cuFFT plan transforms at once
  double2* spec = nullptr;  // fft_batch * ny * (nx/2 + 1) complex values
};

void obs_free(ObsState* o) {
  if (!o) return;
  if (o->part) cudaFree(o->part);
  if (o->fft_ok) cufftDestroy(o->fft);
  if (o->spec) cudaFree(o->spec);
  delete o;
}

}  // namespace chx

using namespace chx;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 304;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of NV values; thread 0 writes them to out[0..NV).
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* out) {
  __shared__ double s[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    v[k] = warp_sum(v[k]);
    if (lane == 0) s[k][wid] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0;
      for (int w = 0; w < kThreads / 32; ++w) a += s[k][w];
      out[k] = a;
    }
  }
}

__device__ __forceinline__ double simpson_w(int i, int n) {
  return (n & 1) ? 1.0 : ((i & 1) ? 4.0 / 3.0 : 2.0 / 3.0);
}

// Slot z = blockIdx.y of G fields of nx*ny; gls[z] = gamma_z / dx^2, rho = dx^2 / dy^2.
__global__ void __launch_bounds__(kThreads) obs_partial_kernel(const double* __restrict__ c, int nx, int ny,
                                                               const double* __restrict__ gls, double rho,
                                                               double* __restrict__ part) {
  const int z = blockIdx.y, nb = gridDim.x;
  const size_t N = (size_t)nx * ny;
  c += (size_t)z * N;
  const double hx = 0.5 * gls[z], hy = hx * rho;
  double v4[4] = {0, 0, 0, 0};  // sum C, energy density, Simpson-weighted C^2, non-finite count
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)nb * blockDim.x) {
    const int j = (int)(p / nx), i = (int)(p - (size_t)j * nx);
    const double v = c[p];
    const double ve = c[(size_t)j * nx + (i + 1 == nx ? 0 : i + 1)];
    const double vn = c[(size_t)(j + 1 == ny ? 0 : j + 1) * nx + i];
    const double q = fma(v, v, -1.0);
    const double gx = ve - v, gy = vn - v;
    v4[0] += v;
    v4[1] += 0.25 * q * q + hx * gx * gx + hy * gy * gy;
    v4[2] += simpson_w(i, nx) * simpson_w(j, ny) * v * v;
    if (!isfinite(v)) v4[3] += 1.0;
  }
  block_sums<4>(v4, part + ((size_t)z * nb + blockIdx.x) * 4);
}

// One thread per slot: out[4 z + 0..2] = mass, F_h, s; out[4 z + 3] = NaN (k1 not formed here).
__global__ void obs_final_kernel(const double* __restrict__ part, int nb, int G, double cell, double inv_np,
                                 double* __restrict__ out, int* status) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= G) return;
  double a[4] = {0, 0, 0, 0};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 4; ++k) a[k] += part[((size_t)z * nb + b) * 4 + k];
  out[4 * z + 0] = a[0] * cell;
  out[4 * z + 1] = a[1] * cell;
  out[4 * z + 2] = 1.0 / (1.0 - a[2] * inv_np);
  out[4 * z + 3] = __longlong_as_double(0x7ff8000000000000ll);
  if (a[3] != 0.0 || !isfinite(a[0]) || !isfinite(a[1])) set_status(status, CHX_ENONFINITE);
}

// Spectral sums over the half spectrum of a real-to-complex transform
// (mx = 0 .. nx/2, my = 0 .. ny-1); modes mx in (0, nx/2) stand for their
// conjugates too.  kx0 = 2 pi / lx, ky0 = 2 pi / ly.
__global__ void __launch_bounds__(kThreads) k1_partial_kernel(const double2* __restrict__ spec, int nx, int ny,
                                                              double kx0, double ky0, double* __restrict__ part) {
  const int nh = nx / 2 + 1;
  const size_t total = (size_t)ny * nh;
  spec += (size_t)blockIdx.y * total;  // field z = blockIdx.y
  part += (size_t)blockIdx.y * gridDim.x * 2;
  double v2[2] = {0, 0};
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / nh), mx = (int)(q - (size_t)j * nh);
    const int my = j <= ny / 2 ? j : j - ny;
    if (mx == 0 && my == 0) continue;
    const double w = (mx == 0 || 2 * mx == nx) ? 1.0 : 2.0;
    const double2 h = spec[q];
    const double pw = w * fma(h.x, h.x, h.y * h.y);
    const double kk = sqrt(kx0 * kx0 * mx * mx + ky0 * ky0 * (double)my * my);
    v2[0] += pw;
    v2[1] += pw / kk;
  }
  block_sums<2>(v2, part + (size_t)blockIdx.x * 2);
}

// One thread per field: out[4 z + 3] = k1 of field z.
__global__ void k1_final_kernel(const double* __restrict__ part, int nb, int G, double* __restrict__ out) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= G) return;
  double num = 0, den = 0;
  for (int b = 0; b < nb; ++b) {
    num += part[((size_t)z * nb + b) * 2];
    den += part[((size_t)z * nb + b) * 2 + 1];
  }
  out[4 * z + 3] = num / den;
}

int blocks_per_slot(size_t N, int G) {
  size_t nb = (N + (size_t)kThreads * 8 - 1) / ((size_t)kThreads * 8);
  if (nb > kMaxBlocks) nb = kMaxBlocks;
  if (G > 1 && nb * G > 65535) nb = 65535 / G;
  return nb < 1 ? 1 : (int)nb;
}

int ensure_part(ObsState* o, size_t doubles) {
  if (o->part_cap >= doubles) return CHX_OK;
  if (o->part) cudaFree(o->part);
  o->part = nullptr;
  o->part_cap = 0;
  if (cudaMalloc(&o->part, doubles * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    o->part = nullptr;
    return fail(CHX_ENOMEM, "observables: partial-sum buffer");
  }
  o->part_cap = doubles;
  return CHX_OK;
}

}  // namespace

namespace chx {

int group_observables(ChGroup* g, int gact, const double* fields, double* out, int with_k1, int* status,
                      cudaStream_t st) {
  if (!g->obs) g->obs = new ObsState();
  ObsState* o = g->obs;
  const int nx = g->nx, ny = g->ny;
  const size_t N = (size_t)nx * ny;
  const int nb = blocks_per_slot(N, gact);
  const int kb = blocks_per_slot((size_t)ny * (nx / 2 + 1), gact);
  // one partial-sum buffer, sized before any launch that uses it
  const size_t need_obs = (size_t)gact * nb * 4, need_k1 = with_k1 ? (size_t)gact * kb * 2 : 0;
  int rc = ensure_part(o, need_obs > need_k1 ? need_obs : need_k1);
  if (rc) return rc;
  obs_partial_kernel<<<dim3(nb, gact), kThreads, 0, st>>>(fields, nx, ny, g->d_gl, g->rho, o->part);
  obs_final_kernel<<<ceil_div(gact, 128), 128, 0, st>>>(o->part, nb, gact, g->dx * g->dy, 1.0 / (double)N, out,
                                                        status);
  rc = launch_check("observables");
  if (rc || !with_k1) return rc;
  if (!o->fft_ok || o->fft_batch != gact) {
    if (o->fft_ok) cufftDestroy(o->fft);
    o->fft_ok = false;
    if (o->spec) cudaFree(o->spec);
    o->spec = nullptr;
    int dims[2] = {ny, nx};
    if (cufftPlanMany(&o->fft, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_D2Z, gact) != CUFFT_SUCCESS)
      return fail(CHX_ENOMEM, "observables: cuFFT plan %d x %d x %d", gact, ny, nx);
    o->fft_ok = true;
    o->fft_batch = gact;
    if (cudaMalloc(&o->spec, (size_t)gact * ny * (nx / 2 + 1) * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      o->spec = nullptr;
      cufftDestroy(o->fft);
      o->fft_ok = false;
      return fail(CHX_ENOMEM, "observables: spectrum buffer");
    }
  }
  if (cufftSetStream(o->fft, st) != CUFFT_SUCCESS ||
      cufftExecD2Z(o->fft, const_cast<double*>(fields), reinterpret_cast<cufftDoubleComplex*>(o->spec)) !=
          CUFFT_SUCCESS)
    return fail(CHX_ECUDA, "observables: cuFFT transform");
  k1_partial_kernel<<<dim3(kb, gact), kThreads, 0, st>>>(o->spec, nx, ny, 2.0 * M_PI / g->lx, 2.0 * M_PI / g->ly,
                                                         o->part);
  k1_final_kernel<<<ceil_div(gact, 128), 128, 0, st>>>(o->part, kb, gact, out);
  return launch_check("observables: k1");
}

}  // namespace chx
