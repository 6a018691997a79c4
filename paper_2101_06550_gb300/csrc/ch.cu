// Semi-implicit ADI step of the periodic 2D Cahn-Hilliard equation (Eq. 3.1)
// and its mass / free-energy diagnostics.
//
// Per step (FP64):
//   rhs      stencil pass: r = -(2/3)(C^n - C^{n-1}) + (2/3) dt Lap_h M,
//            M = (C^n)^3 - C^n - gamma Lap_h Cbar, Cbar = 2C^n - C^{n-1}.
//            The 13-point biharmonic of the paper is applied as Lap_h(Lap_h .)
//            (the two are the same operator: (dxx + dyy)^2 = dxxxx + 2 dxxyy
//            + dyyyy), so both the linear and the nonlinear term go through
//            one 5-point Laplacian of M.  r is written transposed so the row
//            systems of the x sweep become interleaved (coalesced).
//   x sweep  (I + a_x d_xxxx) w = r along rows; y sweep (I + a_y d_yyyy) v = w
//            along columns; update C^{n+1} = Cbar + v.
// Each sweep splits every cyclic system into P segments (a partitioned,
// SPIKE-type solve) so a single grid gives n * P independent threads instead
// of the paper's n: segment-local LU sweeps (the paper's factor/solve steps on
// the shared Toeplitz block), a small reduced system for the 4 boundary
// unknowns of each segment (inverse precomputed on the host in FP64, like the
// paper's precomputed 2x2 bordering inverse), then the spike correction
// x = y - V t_{s+1} - W b_{s-1}, fused into the next pass.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include "chx_internal.cuh"

using namespace chx;

namespace {

struct SpikeDir {
  int n = 0, P = 1, m = 0, nsys = 0;
  double a = 0, b = 0, c = 0;   // LHS row (a, b, c, b, a)
  double* d_lu = nullptr;       // 4*m: ralpha, beta, gam, del of the segment block
  double* d_vw = nullptr;       // 4*m: V0, V1, W0, W1
  double* d_rinv = nullptr;     // (4P)^2
  float* d_lu32 = nullptr;
  float* d_vw32 = nullptr;
  float* d_rinv32 = nullptr;
};

}  // namespace

struct chx_ch_plan {
  PlanHdr hdr;
  int nx, ny, precision;
  double lx, ly, gamma, dt, dx, dy;
  double rho, kap, gl, k1, k2;  // stencil constants
  SpikeDir X, Y;
  double* d_partials;
  int npart;
  // work layout (byte offsets into the caller's work buffer)
  size_t off_f, off_w, off_y1, off_y2, off_ybx, off_tx, off_ybx2, off_tx2, off_yby, off_ty, off_yby2, off_ty2;
  size_t work_bytes;
  // optional per-kernel event timing (ch_profile)
  int prof_on;
  std::vector<cudaEvent_t>* ev_pool;
  std::vector<int>* pend_slot;                      // slot of each pending pair
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* pend;
  double prof_ms[16];
  long long prof_n[16];
};

namespace {

enum Slot { kRhs, kLocX, kRedX, kRefX, kRed2X, kFinX, kLocY, kRedY, kRefY, kRed2Y, kUpd, kSlots };
const char* const kSlotName[kSlots] = {"ch_rhs",         "spike_local_x", "spike_reduced_x", "spike_refine_x",
                                       "spike_reduced2_x", "ch_xfinish",   "spike_local_y",   "spike_reduced_y",
                                       "spike_refine_y", "spike_reduced2_y", "ch_update"};

constexpr int kT = 32;      // tile edge of the transposing kernels
constexpr int kBY = 8;      // tile threads in y
constexpr int kSolveThreads = 128;

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// RHS stencil pass.  Tile of 32 (i) x 32 (j) outputs, Cn/Cbar staged with a
// 2-point halo, M with a 1-point halo.  TC: arithmetic type, TO: output type.
template <typename TC, typename TO>
__global__ void __launch_bounds__(kT* kBY) ch_rhs_kernel(const double* __restrict__ cn, const double* __restrict__ cp,
                                                         TO* __restrict__ rT, int nx, int ny, TC rho, TC kap, TC gl,
                                                         TC k1, TC k2) {
  __shared__ TC s_cn[kT + 4][kT + 5];
  __shared__ TC s_cb[kT + 4][kT + 5];
  __shared__ TC s_m[kT + 2][kT + 3];
  __shared__ TO s_o[kT][kT + 1];
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int tid = threadIdx.y * kT + threadIdx.x;
  for (int idx = tid; idx < (kT + 4) * (kT + 4); idx += kT * kBY) {
    const int ly = idx / (kT + 4), lx = idx % (kT + 4);
    const int gi = wrapi(i0 - 2 + lx, nx), gj = wrapi(j0 - 2 + ly, ny);
    const size_t p = (size_t)gj * nx + gi;
    const TC a = (TC)cn[p], b = (TC)cp[p];
    s_cn[ly][lx] = a;
    s_cb[ly][lx] = fma(TC(2), a, -b);
  }
  __syncthreads();
  for (int idx = tid; idx < (kT + 2) * (kT + 2); idx += kT * kBY) {
    const int ly = idx / (kT + 2) + 1, lx = idx % (kT + 2) + 1;
    TC l = s_cb[ly][lx - 1] + s_cb[ly][lx + 1];
    l = fma(rho, s_cb[ly - 1][lx] + s_cb[ly + 1][lx], l);
    l = fma(kap, s_cb[ly][lx], l);
    const TC c = s_cn[ly][lx];
    const TC nl = c * fma(c, c, TC(-1));
    s_m[ly - 1][lx - 1] = fma(-gl, l, nl);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int ly = threadIdx.y + k * kBY + 1, lx = threadIdx.x + 1;
    TC l = s_m[ly][lx - 1] + s_m[ly][lx + 1];
    l = fma(rho, s_m[ly - 1][lx] + s_m[ly + 1][lx], l);
    l = fma(kap, s_m[ly][lx], l);
    const TC diff = s_cb[ly + 1][lx + 1] - s_cn[ly + 1][lx + 1];  // C^n - C^{n-1}
    s_o[lx - 1][ly - 1] = (TO)fma(k2, l, -(k1 * diff));
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int li = threadIdx.y + k * kBY, lj = threadIdx.x;
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) rT[(size_t)gi * ny + gj] = s_o[li][lj];
  }
}

// ---------------------------------------------------------------------------
// Segment-local LU sweeps on interleaved data: element r of segment s of
// system j at [(s*m + r)*ld + j].  Writes y = A_seg^{-1} f and the four
// boundary values (y_0, y_1, y_{m-2}, y_{m-1}) of every segment.
template <typename TIn, typename TC>
__global__ void __launch_bounds__(kSolveThreads) spike_local_kernel(const TIn* f, TC* y, int ld, int nsys, int m,
                                                                    TC a, const TC* __restrict__ lu, TC* __restrict__ yb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int s = blockIdx.y;
  const size_t L = (size_t)ld;
  const TIn* pf = f + (size_t)s * m * L + j;
  TC* py = y + (size_t)s * m * L + j;
  const TC *ra = lu, *be = lu + m, *ga = lu + 2 * m, *de = lu + 3 * m;
  constexpr int U = 8;
  TC g1 = 0, g2 = 0;
  TC buf[U];
#pragma unroll
  for (int u = 0; u < U; ++u) buf[u] = (u < m) ? (TC)pf[(size_t)u * L] : TC(0);
  for (int r0 = 0; r0 < m; r0 += U) {
    TC nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + U + u;
      nxt[u] = (r < m) ? (TC)pf[(size_t)r * L] : TC(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r < m) {
        TC g = fma(-a, g2, buf[u]);
        g = fma(-__ldg(&be[r]), g1, g) * __ldg(&ra[r]);
        py[(size_t)r * L] = g;
        g2 = g1;
        g1 = g;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) buf[u] = nxt[u];
  }
  TC x1 = 0, x2 = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int r = m - 1 - u;
    buf[u] = (r >= 0) ? py[(size_t)r * L] : TC(0);
  }
  TC ylast = 0, ylast2 = 0;
  for (int r0 = m - 1; r0 >= 0; r0 -= U) {
    TC nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - U - u;
      nxt[u] = (r >= 0) ? py[(size_t)r * L] : TC(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        TC v = fma(-__ldg(&ga[r]), x1, buf[u]);
        v = fma(-__ldg(&de[r]), x2, v);
        py[(size_t)r * L] = v;
        if (r == m - 1) ylast = v;
        if (r == m - 2) ylast2 = v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) buf[u] = nxt[u];
  }
  const size_t S = (size_t)nsys;
  yb[(size_t)(4 * s + 0) * S + j] = x1;  // y_0
  yb[(size_t)(4 * s + 1) * S + j] = x2;  // y_1
  yb[(size_t)(4 * s + 2) * S + j] = ylast2;
  yb[(size_t)(4 * s + 3) * S + j] = ylast;
}

// Reduced system: tau = Rinv * yb for every system (4P unknowns each).
template <typename TC>
__global__ void __launch_bounds__(kSolveThreads) spike_reduced_kernel(const TC* __restrict__ yb,
                                                                      const TC* __restrict__ rinv,
                                                                      TC* __restrict__ tau, int nsys, int k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int q = blockIdx.y;
  const TC* row = rinv + (size_t)q * k;
  TC acc = 0;
  for (int p = 0; p < k; ++p) acc = fma(__ldg(&row[p]), yb[(size_t)p * nsys + j], acc);
  tau[(size_t)q * nsys + j] = acc;
}

// Spike correction of element (row r of segment s) of system j.
template <typename TC>
__device__ __forceinline__ TC spike_corr(const TC* __restrict__ vw, const TC* __restrict__ tau, int m, int P,
                                         int nsys, int s, int r, int j) {
  const int sn = s + 1 == P ? 0 : s + 1, sp = s == 0 ? P - 1 : s - 1;
  const size_t S = (size_t)nsys;
  TC c = __ldg(&vw[r]) * tau[(size_t)(4 * sn + 0) * S + j];
  c = fma(__ldg(&vw[m + r]), tau[(size_t)(4 * sn + 1) * S + j], c);
  c = fma(__ldg(&vw[2 * m + r]), tau[(size_t)(4 * sp + 2) * S + j], c);
  c = fma(__ldg(&vw[3 * m + r]), tau[(size_t)(4 * sp + 3) * S + j], c);
  return c;
}

// x-sweep correction + transpose back: yT (element i of row-system j at
// yT[i*ny + j]) -> w[j*nx + i].  With two (y, tau) pairs the results add
// (first solution + refinement correction).
template <typename TC, typename TO, bool kTwo>
__global__ void __launch_bounds__(kT* kBY) ch_xfinish_kernel(const TC* __restrict__ y1, const TC* __restrict__ t1,
                                                             const TC* __restrict__ y2, const TC* __restrict__ t2,
                                                             const TC* __restrict__ vw, TO* __restrict__ w, int nx,
                                                             int ny, int m, int P) {
  __shared__ TO s_t[kT][kT + 1];
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int j = j0 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int li = threadIdx.y + k * kBY, i = i0 + li;
    if (i < nx && j < ny) {
      const int s = i / m, r = i - s * m;
      TC v = y1[(size_t)i * ny + j] - spike_corr(vw, t1, m, P, ny, s, r, j);
      if (kTwo) v += y2[(size_t)i * ny + j] - spike_corr(vw, t2, m, P, ny, s, r, j);
      s_t[li][threadIdx.x] = (TO)v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int lj = threadIdx.y + k * kBY, li = threadIdx.x;
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) w[(size_t)gj * nx + gi] = s_t[li][lj];
  }
}

// y-sweep correction + update C^{n+1} = 2C^n - C^{n-1} + v.  keep_roles = 1
// writes C^n into c_prev and C^{n+1} into c_now; otherwise C^{n+1} goes into
// c_prev (the caller swaps the pointers).
template <typename TC, bool kTwo>
__global__ void __launch_bounds__(kSolveThreads) ch_update_kernel(const TC* __restrict__ y1, const TC* __restrict__ t1,
                                                                  const TC* __restrict__ y2, const TC* __restrict__ t2,
                                                                  const TC* __restrict__ vw, double* cn, double* cp,
                                                                  int nx, int ny, int m, int P, int keep_roles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx) return;
  const int s = j / m, r = j - s * m;
  const size_t p = (size_t)j * nx + i;
  TC v = y1[p] - spike_corr(vw, t1, m, P, nx, s, r, i);
  if (kTwo) v += y2[p] - spike_corr(vw, t2, m, P, nx, s, r, i);
  const double a = cn[p], b = cp[p];
  const double nxt = fma(2.0, a, -b) + (double)v;
  if (keep_roles) {
    cp[p] = a;
    cn[p] = nxt;
  } else {
    cp[p] = nxt;
  }
}

// FP32 refinement sweep: residual rho = f - A x0 in FP64 with x0 the corrected
// first FP32 solution (from y1, tau1), then the segment-local FP32 LU sweeps on
// rho into y2, plus the boundary values for the second reduced solve.
__device__ __forceinline__ double x0_at(const float* __restrict__ y1, const float* __restrict__ t1,
                                        const float* __restrict__ vw, int n, int m, int P, int ld, int nsys, int i,
                                        int j) {
  i = wrapi(i, n);
  const int s = i / m, r = i - s * m;
  return (double)(y1[(size_t)i * ld + j] - spike_corr(vw, t1, m, P, nsys, s, r, j));
}

__global__ void __launch_bounds__(kSolveThreads) spike_refine_kernel(
    const float* __restrict__ f, const float* __restrict__ y1, const float* __restrict__ t1, float* __restrict__ y2,
    float* __restrict__ yb, int ld, int nsys, int n, int m, int P, double ca, double cb, double cc, float a32,
    const float* __restrict__ lu, const float* __restrict__ vw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int s = blockIdx.y;
  const int base = s * m;
  const size_t L = (size_t)ld;
  const float *ra = lu, *be = lu + m, *ga = lu + 2 * m, *de = lu + 3 * m;
  double w0 = x0_at(y1, t1, vw, n, m, P, ld, nsys, base - 2, j);
  double w1 = x0_at(y1, t1, vw, n, m, P, ld, nsys, base - 1, j);
  double w2 = x0_at(y1, t1, vw, n, m, P, ld, nsys, base, j);
  double w3 = x0_at(y1, t1, vw, n, m, P, ld, nsys, base + 1, j);
  double w4 = x0_at(y1, t1, vw, n, m, P, ld, nsys, base + 2, j);
  float g1 = 0.f, g2 = 0.f;
  for (int r = 0; r < m; ++r) {
    const int i = base + r;
    double ax = cc * w2;
    ax = fma(cb, w1 + w3, ax);
    ax = fma(ca, w0 + w4, ax);
    const float res = (float)((double)f[(size_t)i * L + j] - ax);
    float g = fmaf(-a32, g2, res);
    g = fmaf(-__ldg(&be[r]), g1, g) * __ldg(&ra[r]);
    y2[(size_t)i * L + j] = g;
    g2 = g1;
    g1 = g;
    w0 = w1; w1 = w2; w2 = w3; w3 = w4;
    w4 = x0_at(y1, t1, vw, n, m, P, ld, nsys, i + 3, j);
  }
  float x1 = 0.f, x2 = 0.f, ylast = 0.f, ylast2 = 0.f;
  for (int r = m - 1; r >= 0; --r) {
    const size_t p = (size_t)(base + r) * L + j;
    float v = fmaf(-__ldg(&ga[r]), x1, y2[p]);
    v = fmaf(-__ldg(&de[r]), x2, v);
    y2[p] = v;
    if (r == m - 1) ylast = v;
    if (r == m - 2) ylast2 = v;
    x2 = x1;
    x1 = v;
  }
  const size_t S = (size_t)nsys;
  yb[(size_t)(4 * s + 0) * S + j] = x1;
  yb[(size_t)(4 * s + 1) * S + j] = x2;
  yb[(size_t)(4 * s + 2) * S + j] = ylast2;
  yb[(size_t)(4 * s + 3) * S + j] = ylast;
}

// ---------------------------------------------------------------------------
// Diagnostics: per-block partial sums (fixed order), then one block.
constexpr int kDiagBlocks = 304, kDiagThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kDiagThreads) ch_diag_partial_kernel(const double* __restrict__ c, int nx, int ny,
                                                                       double half_gamma_ix2, double half_gamma_iy2,
                                                                       double* __restrict__ part) {
  double sm = 0.0, se = 0.0, bad = 0.0;
  const size_t N = (size_t)nx * ny;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(p / nx), i = (int)(p - (size_t)j * nx);
    const double v = c[p];
    const double ve = c[(size_t)j * nx + (i + 1 == nx ? 0 : i + 1)];
    const double vn = c[(size_t)(j + 1 == ny ? 0 : j + 1) * nx + i];
    const double q = fma(v, v, -1.0);
    const double gx = ve - v, gy = vn - v;
    sm += v;
    se += 0.25 * q * q + half_gamma_ix2 * gx * gx + half_gamma_iy2 * gy * gy;
    if (!isfinite(v)) bad = 1.0;
  }
  __shared__ double s[3][kDiagThreads / 32];
  sm = warp_sum(sm);
  se = warp_sum(se);
  bad = warp_sum(bad);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s[0][wid] = sm; s[1][wid] = se; s[2][wid] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0;
    for (int w = 0; w < kDiagThreads / 32; ++w) { a += s[0][w]; b += s[1][w]; d += s[2][w]; }
    part[3 * blockIdx.x + 0] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = d;
  }
}

__global__ void ch_diag_final_kernel(const double* __restrict__ part, int nb, double cell, double* mass,
                                     double* energy, int* status) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0, d = 0;
  for (int k = 0; k < nb; ++k) { a += part[3 * k]; b += part[3 * k + 1]; d += part[3 * k + 2]; }
  *mass = a * cell;
  *energy = b * cell;
  if (d != 0.0 || !isfinite(a) || !isfinite(b)) set_status(status, CHX_ENONFINITE);
}

// ---------------------------------------------------------------------------
// Host: segment count and precomputation for one sweep direction.
int choose_segments(int n, int nsys) {
  int pmax = (int)floor(sqrt(n / 8.0));
  if (pmax < 1) pmax = 1;
  int want = (32768 + nsys - 1) / nsys;
  if (want < 1) want = 1;
  int lim = pmax < want ? pmax : want;
  for (int P = lim; P >= 1; --P)
    if (n % P == 0 && n / P >= 8) return P;
  return 1;
}

template <typename T>
int dev_upload(T** dst, const std::vector<double>& src) {
  std::vector<T> h(src.size());
  for (size_t i = 0; i < src.size(); ++i) h[i] = (T)src[i];
  if (cudaMalloc(dst, h.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return fail(CHX_ENOMEM, "ch_plan_create: allocation of %zu values", h.size());
  }
  return cuda_check(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "ch_plan_create: upload");
}

int setup_dir(SpikeDir* D, int n, int nsys, double acoef) {
  D->n = n;
  D->nsys = nsys;
  D->a = acoef;
  D->b = -4.0 * acoef;
  D->c = 1.0 + 6.0 * acoef;
  D->P = choose_segments(n, nsys);
  D->m = n / D->P;
  const int m = D->m, P = D->P, k = 4 * P;
  std::vector<double> lu(4 * (size_t)m), vw(4 * (size_t)m), R((size_t)k * k, 0.0), Rinv((size_t)k * k);
  double *ra = &lu[0], *be = &lu[m], *ga = &lu[2 * (size_t)m], *de = &lu[3 * (size_t)m];
  int rc = band_factor_host(m, D->a, D->b, D->c, D->b, D->a, ra, be, ga, de);
  if (rc) return rc;
  // V = A_seg^{-1} [e at row m-2; d, e at row m-1] (couples t_{s+1}),
  // W = A_seg^{-1} [a, b at row 0; 0, a at row 1] (couples b_{s-1}).
  std::vector<double> rhs(m), col(m);
  for (int q = 0; q < 4; ++q) {
    std::fill(rhs.begin(), rhs.end(), 0.0);
    if (q < 2) {
      rhs[m - 2] += q == 0 ? D->a : 0.0;   // e = a
      rhs[m - 1] += q == 0 ? D->b : D->a;  // d = b, e = a
    } else {
      rhs[0] += q == 2 ? D->a : D->b;      // a, b
      rhs[1] += q == 2 ? 0.0 : D->a;       // 0, a
    }
    band_solve_host(m, D->a, ra, be, ga, de, rhs.data(), col.data());
    for (int r = 0; r < m; ++r) vw[(size_t)q * m + r] = col[r];
  }
  const int rows[4] = {0, 1, m - 2, m - 1};
  for (int s = 0; s < P; ++s) {
    const int sn = (s + 1) % P, sp = (s - 1 + P) % P;
    for (int q = 0; q < 4; ++q) {
      const int r = rows[q], row = 4 * s + q;
      R[(size_t)row * k + row] += 1.0;
      R[(size_t)row * k + 4 * sn + 0] += vw[0 * (size_t)m + r];
      R[(size_t)row * k + 4 * sn + 1] += vw[1 * (size_t)m + r];
      R[(size_t)row * k + 4 * sp + 2] += vw[2 * (size_t)m + r];
      R[(size_t)row * k + 4 * sp + 3] += vw[3 * (size_t)m + r];
    }
  }
  rc = dense_inverse_host(k, R.data(), Rinv.data());
  if (rc) return rc;
  if ((rc = dev_upload(&D->d_lu, lu)) || (rc = dev_upload(&D->d_vw, vw)) || (rc = dev_upload(&D->d_rinv, Rinv)) ||
      (rc = dev_upload(&D->d_lu32, lu)) || (rc = dev_upload(&D->d_vw32, vw)) || (rc = dev_upload(&D->d_rinv32, Rinv)))
    return rc;
  return CHX_OK;
}

void free_dir(SpikeDir* D) {
  cudaFree(D->d_lu); cudaFree(D->d_vw); cudaFree(D->d_rinv);
  cudaFree(D->d_lu32); cudaFree(D->d_vw32); cudaFree(D->d_rinv32);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

namespace chx {
void ch_plan_free(chx_ch_plan* p) {
  if (!p) return;
  free_dir(&p->X);
  free_dir(&p->Y);
  if (p->d_partials) cudaFree(p->d_partials);
  if (p->pend) {
    for (auto& e : *p->pend) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    delete p->pend;
  }
  if (p->ev_pool) {
    for (auto e : *p->ev_pool) cudaEventDestroy(e);
    delete p->ev_pool;
  }
  delete p->pend_slot;
  hdr_free(&p->hdr);
  free(p);
}
}  // namespace chx

extern "C" int ch_plan_create(chx_ch_plan** plan, int nx, int ny, double lx, double ly, double gamma, double dt,
                              int precision) {
  if (!plan) return fail(CHX_EINVAL, "ch_plan_create: null plan pointer");
  *plan = nullptr;
  if (nx < 8 || ny < 8 || nx > 16384 || ny > 16384)
    return fail(CHX_EINVAL, "ch_plan_create: nx %d, ny %d outside [8, 16384]", nx, ny);
  if (!(lx > 0) || !(ly > 0) || !(dt > 0) || !(gamma >= 0) || !isfinite(lx) || !isfinite(ly) || !isfinite(dt) ||
      !isfinite(gamma))
    return fail(CHX_EINVAL, "ch_plan_create: lx %g, ly %g, dt %g, gamma %g", lx, ly, dt, gamma);
  if (precision != CHX_PREC_F64 && precision != CHX_PREC_F32_REFINE)
    return fail(CHX_EINVAL, "ch_plan_create: precision %d", precision);
  chx_ch_plan* p = (chx_ch_plan*)calloc(1, sizeof(chx_ch_plan));
  if (!p) return fail(CHX_ENOMEM, "ch_plan_create: plan allocation");
  new (&p->X) SpikeDir();
  new (&p->Y) SpikeDir();
  p->ev_pool = new std::vector<cudaEvent_t>();
  p->pend = new std::vector<std::pair<cudaEvent_t, cudaEvent_t>>();
  p->pend_slot = new std::vector<int>();
  int rc = hdr_init(&p->hdr, kMagicCh);
  if (rc) { ch_plan_free(p); return rc; }
  p->nx = nx; p->ny = ny; p->precision = precision;
  p->lx = lx; p->ly = ly; p->gamma = gamma; p->dt = dt;
  p->dx = lx / nx; p->dy = ly / ny;
  const double sx = 1.0 / (p->dx * p->dx);
  p->rho = (p->dx * p->dx) / (p->dy * p->dy);
  p->kap = -2.0 * (1.0 + p->rho);
  p->gl = gamma * sx;
  p->k1 = 2.0 / 3.0;
  p->k2 = (2.0 / 3.0) * dt * sx;
  const double ax = (2.0 / 3.0) * gamma * dt / (p->dx * p->dx * p->dx * p->dx);
  const double ay = (2.0 / 3.0) * gamma * dt / (p->dy * p->dy * p->dy * p->dy);
  if ((rc = setup_dir(&p->X, nx, ny, ax)) || (rc = setup_dir(&p->Y, ny, nx, ay))) { ch_plan_free(p); return rc; }
  p->npart = kDiagBlocks;
  if (cudaMalloc(&p->d_partials, 3 * (size_t)kDiagBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    p->d_partials = nullptr;
    ch_plan_free(p);
    return fail(CHX_ENOMEM, "ch_plan_create: diagnostics scratch");
  }
  const size_t N = (size_t)nx * ny;
  const size_t esz = precision == CHX_PREC_F64 ? 8 : 4;
  size_t off = 0;
  p->off_f = off; off = align256(off + N * esz);
  p->off_w = off; off = align256(off + N * esz);
  p->off_y1 = off; off = align256(off + (precision == CHX_PREC_F64 ? 0 : N * esz));
  p->off_y2 = off; off = align256(off + (precision == CHX_PREC_F64 ? 0 : N * esz));
  const size_t kx = 4 * (size_t)p->X.P * ny, ky = 4 * (size_t)p->Y.P * nx;
  p->off_ybx = off; off = align256(off + kx * esz);
  p->off_tx = off; off = align256(off + kx * esz);
  p->off_ybx2 = off; off = align256(off + kx * esz);
  p->off_tx2 = off; off = align256(off + kx * esz);
  p->off_yby = off; off = align256(off + ky * esz);
  p->off_ty = off; off = align256(off + ky * esz);
  p->off_yby2 = off; off = align256(off + ky * esz);
  p->off_ty2 = off; off = align256(off + ky * esz);
  p->work_bytes = off;
  *plan = p;
  return CHX_OK;
}

extern "C" size_t ch_work_bytes(const chx_ch_plan* p) {
  if (!p || p->hdr.magic != kMagicCh) return 0;
  return p->work_bytes;
}

static cudaEvent_t prof_event(chx_ch_plan* p) {
  if (!p->ev_pool->empty()) {
    cudaEvent_t e = p->ev_pool->back();
    p->ev_pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events when profiling is on.
struct ProfScope {
  chx_ch_plan* p;
  int slot;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  ProfScope(chx_ch_plan* p_, int slot_, cudaStream_t st_) : p(p_), slot(slot_), st(st_) {
    if (p->prof_on) {
      e0 = prof_event(p);
      cudaEventRecord(e0, st);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEvent_t e1 = prof_event(p);
      cudaEventRecord(e1, st);
      p->pend->push_back({e0, e1});
      p->pend_slot->push_back(slot);
    }
  }
};
#define PROF(slot) ProfScope prof_scope_##slot(p, slot, st)

template <typename T>
static T* wptr(void* work, size_t off) {
  return (T*)((char*)work + off);
}

static void step_f64(chx_ch_plan* p, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st) {
  const int nx = p->nx, ny = p->ny;
  double* f = wptr<double>(work, p->off_f);
  double* w = wptr<double>(work, p->off_w);
  double *ybx = wptr<double>(work, p->off_ybx), *tx = wptr<double>(work, p->off_tx);
  double *yby = wptr<double>(work, p->off_yby), *ty = wptr<double>(work, p->off_ty);
  const dim3 tgrid(ceil_div(nx, kT), ceil_div(ny, kT)), tblock(kT, kBY);
  const SpikeDir &X = p->X, &Y = p->Y;
  const dim3 gx(ceil_div(ny, kSolveThreads), X.P), gy(ceil_div(nx, kSolveThreads), Y.P);
  { PROF(kRhs); ch_rhs_kernel<double, double><<<tgrid, tblock, 0, st>>>(cur, prev, f, nx, ny, p->rho, p->kap, p->gl, p->k1, p->k2); }
  { PROF(kLocX); spike_local_kernel<double, double><<<gx, kSolveThreads, 0, st>>>(f, f, ny, ny, X.m, X.a, X.d_lu, ybx); }
  { PROF(kRedX); spike_reduced_kernel<double><<<dim3(gx.x, 4 * X.P), kSolveThreads, 0, st>>>(ybx, X.d_rinv, tx, ny, 4 * X.P); }
  { PROF(kFinX); ch_xfinish_kernel<double, double, false><<<tgrid, tblock, 0, st>>>(f, tx, nullptr, nullptr, X.d_vw, w, nx, ny, X.m, X.P); }
  { PROF(kLocY); spike_local_kernel<double, double><<<gy, kSolveThreads, 0, st>>>(w, w, nx, nx, Y.m, Y.a, Y.d_lu, yby); }
  { PROF(kRedY); spike_reduced_kernel<double><<<dim3(gy.x, 4 * Y.P), kSolveThreads, 0, st>>>(yby, Y.d_rinv, ty, nx, 4 * Y.P); }
  { PROF(kUpd); ch_update_kernel<double, false><<<dim3(ceil_div(nx, kSolveThreads), ny), kSolveThreads, 0, st>>>(
        w, ty, nullptr, nullptr, Y.d_vw, cur, prev, nx, ny, Y.m, Y.P, keep_roles); }
}

static void step_f32r(chx_ch_plan* p, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st) {
  const int nx = p->nx, ny = p->ny;
  float* f = wptr<float>(work, p->off_f);
  float* w = wptr<float>(work, p->off_w);
  float* y1 = wptr<float>(work, p->off_y1);
  float* y2 = wptr<float>(work, p->off_y2);
  float *ybx = wptr<float>(work, p->off_ybx), *tx = wptr<float>(work, p->off_tx);
  float *ybx2 = wptr<float>(work, p->off_ybx2), *tx2 = wptr<float>(work, p->off_tx2);
  float *yby = wptr<float>(work, p->off_yby), *ty = wptr<float>(work, p->off_ty);
  float *yby2 = wptr<float>(work, p->off_yby2), *ty2 = wptr<float>(work, p->off_ty2);
  const dim3 tgrid(ceil_div(nx, kT), ceil_div(ny, kT)), tblock(kT, kBY);
  const SpikeDir &X = p->X, &Y = p->Y;
  const dim3 gx(ceil_div(ny, kSolveThreads), X.P), gy(ceil_div(nx, kSolveThreads), Y.P);
  { PROF(kRhs); ch_rhs_kernel<float, float><<<tgrid, tblock, 0, st>>>(cur, prev, f, nx, ny, (float)p->rho, (float)p->kap,
                                                        (float)p->gl, (float)p->k1, (float)p->k2); }
  // x: first FP32 solve, FP64-residual refinement, combine + transpose.
  { PROF(kLocX); spike_local_kernel<float, float><<<gx, kSolveThreads, 0, st>>>(f, y1, ny, ny, X.m, (float)X.a, X.d_lu32, ybx); }
  { PROF(kRedX); spike_reduced_kernel<float><<<dim3(gx.x, 4 * X.P), kSolveThreads, 0, st>>>(ybx, X.d_rinv32, tx, ny, 4 * X.P); }
  { PROF(kRefX); spike_refine_kernel<<<gx, kSolveThreads, 0, st>>>(f, y1, tx, y2, ybx2, ny, ny, nx, X.m, X.P, X.a, X.b, X.c,
                                                    (float)X.a, X.d_lu32, X.d_vw32); }
  { PROF(kRed2X); spike_reduced_kernel<float><<<dim3(gx.x, 4 * X.P), kSolveThreads, 0, st>>>(ybx2, X.d_rinv32, tx2, ny, 4 * X.P); }
  { PROF(kFinX); ch_xfinish_kernel<float, float, true><<<tgrid, tblock, 0, st>>>(y1, tx, y2, tx2, X.d_vw32, w, nx, ny, X.m, X.P); }
  // y
  { PROF(kLocY); spike_local_kernel<float, float><<<gy, kSolveThreads, 0, st>>>(w, y1, nx, nx, Y.m, (float)Y.a, Y.d_lu32, yby); }
  { PROF(kRedY); spike_reduced_kernel<float><<<dim3(gy.x, 4 * Y.P), kSolveThreads, 0, st>>>(yby, Y.d_rinv32, ty, nx, 4 * Y.P); }
  { PROF(kRefY); spike_refine_kernel<<<gy, kSolveThreads, 0, st>>>(w, y1, ty, y2, yby2, nx, nx, ny, Y.m, Y.P, Y.a, Y.b, Y.c,
                                                    (float)Y.a, Y.d_lu32, Y.d_vw32); }
  { PROF(kRed2Y); spike_reduced_kernel<float><<<dim3(gy.x, 4 * Y.P), kSolveThreads, 0, st>>>(yby2, Y.d_rinv32, ty2, nx, 4 * Y.P); }
  { PROF(kUpd); ch_update_kernel<float, true><<<dim3(ceil_div(nx, kSolveThreads), ny), kSolveThreads, 0, st>>>(
        y1, ty, y2, ty2, Y.d_vw32, cur, prev, nx, ny, Y.m, Y.P, keep_roles); }
}

extern "C" int ch_step(chx_ch_plan* p, double* c_now, double* c_prev, void* work, int nsteps, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_step: bad plan");
  if (!c_now || !c_prev || !work) return fail(CHX_EINVAL, "ch_step: null pointer");
  if (nsteps < 0) return fail(CHX_EINVAL, "ch_step: nsteps %d < 0", nsteps);
  if (((uintptr_t)work & 255) != 0) return fail(CHX_EINVAL, "ch_step: work must be 256-byte aligned");
  const size_t fb = (size_t)p->nx * p->ny * sizeof(double);
  const char *a = (const char*)c_now, *b = (const char*)c_prev, *w = (const char*)work;
  if ((a < b + fb && b < a + fb) || (a < w + p->work_bytes && w < a + fb) || (b < w + p->work_bytes && w < b + fb))
    return fail(CHX_EINVAL, "ch_step: c_now, c_prev and work must not overlap");
  cudaStream_t st = (cudaStream_t)stream;
  double *cur = c_now, *prev = c_prev;
  for (int s = 0; s < nsteps; ++s) {
    const int last = s == nsteps - 1;
    const int keep = last && cur == c_now;
    if (p->precision == CHX_PREC_F64) step_f64(p, cur, prev, work, keep, st);
    else step_f32r(p, cur, prev, work, keep, st);
    if (!keep) {
      double* t = cur;
      cur = prev;
      prev = t;
    }
    int rc = launch_check("ch_step");
    if (rc) return rc;
  }
  p->hdr.last_stream = st;
  return CHX_OK;
}

extern "C" int ch_diagnostics(chx_ch_plan* p, const double* c, double* mass_out, double* energy_out, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_diagnostics: bad plan");
  if (!c || !mass_out || !energy_out) return fail(CHX_EINVAL, "ch_diagnostics: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const double hx = 0.5 * p->gamma / (p->dx * p->dx), hy = 0.5 * p->gamma / (p->dy * p->dy);
  ch_diag_partial_kernel<<<kDiagBlocks, kDiagThreads, 0, st>>>(c, p->nx, p->ny, hx, hy, p->d_partials);
  ch_diag_final_kernel<<<1, 32, 0, st>>>(p->d_partials, kDiagBlocks, p->dx * p->dy, mass_out, energy_out,
                                         p->hdr.d_status);
  p->hdr.last_stream = st;
  return launch_check("ch_diagnostics");
}

extern "C" int ch_profile(chx_ch_plan* p, int enable) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_profile: bad plan");
  p->prof_on = enable ? 1 : 0;
  return CHX_OK;
}

extern "C" int ch_profile_read(chx_ch_plan* p, double* ms, long long* launches, int max_slots, int reset) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_profile_read: bad plan");
  for (size_t k = 0; k < p->pend->size(); ++k) {
    auto& e = (*p->pend)[k];
    int rc = cuda_check(cudaEventSynchronize(e.second), "ch_profile_read: event synchronize");
    if (rc) return rc;
    float t = 0.f;
    cudaEventElapsedTime(&t, e.first, e.second);
    const int slot = (*p->pend_slot)[k];
    p->prof_ms[slot] += t;
    p->prof_n[slot] += 1;
    p->ev_pool->push_back(e.first);
    p->ev_pool->push_back(e.second);
  }
  p->pend->clear();
  p->pend_slot->clear();
  for (int k = 0; k < max_slots && k < kSlots; ++k) {
    if (ms) ms[k] = p->prof_ms[k];
    if (launches) launches[k] = p->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < kSlots; ++k) { p->prof_ms[k] = 0.0; p->prof_n[k] = 0; }
  return kSlots;
}

extern "C" const char* ch_profile_slot_name(int slot) {
  return (slot >= 0 && slot < kSlots) ? kSlotName[slot] : "";
}
