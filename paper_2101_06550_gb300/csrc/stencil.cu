// General 2D stencil apply (cuSten "Compute 2D XY", Sec. 3.3).
//
// Each CTA stages a 32 x 16 output tile plus its halo in shared memory (the
// cuSten block-with-halo design of Sec. 3.2, corner halos included), applying
// the optional pre-map c -> c^3 - c once per loaded value, then every thread
// evaluates the weighted box for two outputs.  Weights travel in the kernel
// parameter block, so the call needs no device allocation.
#include "chx_internal.cuh"

using namespace chx;

namespace {

constexpr int kMaxHalo = 7;
constexpr int kTX = 32, kTY = 16, kBY = 8;
constexpr int kMaxW = (2 * kMaxHalo + 1) * (2 * kMaxHalo + 1);

struct StencilWeights {
  double w[kMaxW];
};

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

template <typename T, bool kPeriodic, bool kPremap>
__global__ void __launch_bounds__(kTX* kBY) stencil_kernel(const T* __restrict__ in, T* __restrict__ out, int nx,
                                                           int ny, int ldx, StencilWeights W, int left, int right,
                                                           int top, int bottom) {
  __shared__ T tile[kTY + 2 * kMaxHalo][kTX + 2 * kMaxHalo + 1];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tw = kTX + left + right, th = kTY + top + bottom;
  for (int ly = threadIdx.y; ly < th; ly += kBY) {
    for (int lx = threadIdx.x; lx < tw; lx += kTX) {
      int gx = x0 - left + lx, gy = y0 - top + ly;
      T v = T(0);
      if (kPeriodic) {
        gx = wrapi(gx, nx);
        gy = wrapi(gy, ny);
        v = in[(size_t)gy * ldx + gx];
      } else if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        v = in[(size_t)gy * ldx + gx];
      }
      if (kPremap) v = v * v * v - v;
      tile[ly][lx] = v;
    }
  }
  __syncthreads();
  const int bw = left + right + 1;
  for (int k = 0; k < kTY / kBY; ++k) {
    const int ty = threadIdx.y + k * kBY, tx = threadIdx.x;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= nx || gy >= ny) continue;
    if (!kPeriodic && (gx - left < 0 || gx + right >= nx || gy - top < 0 || gy + bottom >= ny)) continue;
    T s = T(0);
    for (int dj = 0; dj <= top + bottom; ++dj)
      for (int di = 0; di < bw; ++di) s += (T)W.w[dj * bw + di] * tile[ty + dj][tx + di];
    out[(size_t)gy * ldx + gx] = s;
  }
}

template <typename T>
void launch(const void* in, void* out, int nx, int ny, int ldx, const StencilWeights& W, int l, int r, int t, int b,
            int premap, int periodic, cudaStream_t st) {
  dim3 grid(ceil_div(nx, kTX), ceil_div(ny, kTY)), block(kTX, kBY);
  const T* i = (const T*)in;
  T* o = (T*)out;
  if (periodic) {
    if (premap) stencil_kernel<T, true, true><<<grid, block, 0, st>>>(i, o, nx, ny, ldx, W, l, r, t, b);
    else stencil_kernel<T, true, false><<<grid, block, 0, st>>>(i, o, nx, ny, ldx, W, l, r, t, b);
  } else {
    if (premap) stencil_kernel<T, false, true><<<grid, block, 0, st>>>(i, o, nx, ny, ldx, W, l, r, t, b);
    else stencil_kernel<T, false, false><<<grid, block, 0, st>>>(i, o, nx, ny, ldx, W, l, r, t, b);
  }
}

}  // namespace

extern "C" int stencil_apply_2d(const void* in, void* out, int nx, int ny, int ldx, const double* w_host, int left,
                                int right, int top, int bottom, int premap, int periodic, int dtype, void* stream) {
  if (!in || !out || !w_host) return fail(CHX_EINVAL, "stencil_apply_2d: null pointer");
  if (nx < 1 || ny < 1 || ldx < nx) return fail(CHX_EINVAL, "stencil_apply_2d: nx %d, ny %d, ldx %d", nx, ny, ldx);
  if (left < 0 || right < 0 || top < 0 || bottom < 0 || left > kMaxHalo || right > kMaxHalo || top > kMaxHalo ||
      bottom > kMaxHalo)
    return fail(CHX_EINVAL, "stencil_apply_2d: box extents must lie in [0, %d]", kMaxHalo);
  if (premap != CHX_PREMAP_NONE && premap != CHX_PREMAP_CUBIC_MINUS_C)
    return fail(CHX_EINVAL, "stencil_apply_2d: premap %d", premap);
  if (dtype != CHX_F64 && dtype != CHX_F32) return fail(CHX_EINVAL, "stencil_apply_2d: dtype %d", dtype);
  const size_t esz = dtype == CHX_F64 ? 8 : 4;
  const char* ib = (const char*)in;
  const char* ob = (const char*)out;
  const size_t span = ((size_t)(ny - 1) * ldx + nx) * esz;
  if (ib < ob + span && ob < ib + span) return fail(CHX_EINVAL, "stencil_apply_2d: out must not alias in");
  StencilWeights W;
  const int cnt = (left + right + 1) * (top + bottom + 1);
  for (int k = 0; k < kMaxW; ++k) W.w[k] = k < cnt ? w_host[k] : 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CHX_F64) launch<double>(in, out, nx, ny, ldx, W, left, right, top, bottom, premap, periodic, st);
  else launch<float>(in, out, nx, ny, ldx, W, left, right, top, bottom, premap, periodic, st);
  return launch_check("stencil_apply_2d");
}
