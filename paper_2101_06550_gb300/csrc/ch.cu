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
// Several same-shape simulations run as one group: the stencil, update and y
// sweep index the simulation by blockIdx.z, and the x sweep sees the row
// systems of all of them as one interleaved batch.
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
#include <type_traits>
#include <utility>
#include <vector>

#include "chgroup.cuh"
#include "ff.cuh"
#include "noise.cuh"

using namespace chx;

namespace chx {
const char* const kSlotName[kSlots] = {"ch_rhs",           "spike_local_x",   "spike_reduced_x",  "ch_resid_x",
                                       "spike_local2_x",   "spike_reduced2_x", "ch_xfinish",       "spike_local_y",
                                       "spike_reduced_y",  "ch_resid_y",       "spike_local2_y",   "spike_reduced2_y",
                                       "ch_update",        "ch_rhs_lap",       "x_solve_ff",       "y_solve_ff"};
}  // namespace chx

struct chx_ch_plan {
  PlanHdr hdr;
  ChGroup g;
  double* d_partials;
  Prof* prof;
  // Captured steps, valid for the pointers they were captured with: `pair`
  // (two steps that leave C^n in c_now) and `one` (one role-keeping step).
  cudaGraphExec_t pair, one;
  const void *graph_now, *graph_prev, *graph_work;
  const void *seen_now, *seen_prev, *seen_work;  // the previous call's pointers
  cudaStream_t cap;
  // Cahn-Hilliard-Cook pairs (ch_cook_run): two forced steps whose deviates take
  // their step index from the device counter d_cook_step, valid for these
  // pointers and parameters
  cudaGraphExec_t cook_pair;
  const void *cook_now, *cook_prev, *cook_work, *cook_rho;
  double cook_sigma;
  uint64_t cook_seed, cook_sim;
  uint64_t* d_cook_step;
};

namespace {

constexpr int kT = 32;      // tile edge of the transposing kernels
constexpr int kBY = 8;      // tile threads in y
constexpr int kRBY = 8;     // the RHS passes' threads in y
static_assert(kT * kRBY >= 2 * (kT + 2) && kT % kRBY == 0, "RHS staging assumes one pass over the extra columns");
constexpr int kSolveThreads = 128;
// Rows of the FP64 reduced solve per thread.  Measured at 2048^2 (2048 systems x
// 16 segments per direction), whole graph-replayed step, same box, three rounds:
// 4 rows 0.3082 ms, 2 rows 0.3060 ms, 1 row 0.3068 ms.  Fewer rows per thread
// mean more, shorter single-warp blocks, so the SMs finish closer together
// (with 4 rows ncu showed them idle a quarter of the kernel's time); one row
// per thread loads every boundary value four times.
constexpr int kReducedRows = 2;

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Wrap for indices within a few periods of [0, n): two compares instead of a
// division on the common path.
__device__ __forceinline__ int wrap_near(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  return wrapi(i, n);
}

// ---------------------------------------------------------------------------
// The FP64 right-hand side, in two passes over 32 (i) x 32 (j) tiles of
// simulation blockIdx.z (gls[z] = gamma / dx^2):
//   pass 1 (ch_rhs_m_kernel): Cbar = 2 C^n - C^{n-1} with a 1-point halo, then
//     M = C^3 - C - gamma Lap_h Cbar on the tile; M and Cbar are stored (the
//     update reads Cbar: C^{n+1} = Cbar + v);
//   pass 2 (ch_rhs_r_kernel): r / k2 = Lap_h M - kd (Cbar - C^n), M staged with
//     a 1-point halo, written transposed for the x sweep:
//     rT[i * (G*ny) + z*ny + j].
// A single pass would recompute M on every tile's halo ring (34^2 / 32^2 of
// the points): 15.2 FP64 operations per point against 14.1 here, for one more
// launch and 32 more bytes per point, which these FP64-bound passes absorb.
// r / k2 with k2 = (2/3) dt / dx^2 and kd = dx^2 / dt takes one FMA where r
// itself takes a multiply and an FMA; the solves are linear, so the update
// restores the scale (C^{n+1} = Cbar + k2 v').
// Pass 1's occupancy bound: 8 blocks per SM (32 registers).  Same-box A/B at
// 2048^2: 0.0725 ms per launch, against 0.0727-0.0728 ms with 6 or 4 blocks.
constexpr int kRMMinBlocks = 8;
template <typename TC>
__global__ void __launch_bounds__(kT* kRBY, kRMMinBlocks) ch_rhs_m_kernel(const double* __restrict__ cn,
                                                            const double* __restrict__ cp, double* __restrict__ m,
                                                            double* __restrict__ cbar, int nx, int ny, TC rho,
                                                            TC kap, const TC* __restrict__ gls) {
  __shared__ TC s_cb[kT + 2][kT + 3];
  const int z = blockIdx.z;
  const TC gl = gls[z];
  const size_t off = (size_t)z * nx * ny;
  cn += off;
  cp += off;
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int tid = threadIdx.y * kT + threadIdx.x;
  // whole 32-column rows per warp (bank-conflict free), then the two columns past 32
  auto stage = [&](int ly, int lx) {
    const int gi = wrap_near(i0 - 1 + lx, nx), gj = wrap_near(j0 - 1 + ly, ny);
    const size_t p = (size_t)gj * nx + gi;
    s_cb[ly][lx] = fma(TC(2), (TC)cn[p], -(TC)cp[p]);
  };
#pragma unroll
  for (int k = 0; k < (kT + 2 + kRBY - 1) / kRBY; ++k) {
    const int ly = threadIdx.y + k * kRBY;
    if (ly < kT + 2) stage(ly, threadIdx.x);
  }
  if (tid < 2 * (kT + 2)) stage(tid >> 1, kT + (tid & 1));
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kRBY; ++k) {
    const int ly = 1 + threadIdx.y + k * kRBY, lx = 1 + threadIdx.x;
    const int gi = i0 + threadIdx.x, gj = j0 + ly - 1;
    if (gi < nx && gj < ny) {
      TC l = s_cb[ly][lx - 1] + s_cb[ly][lx + 1];
      l = fma(rho, s_cb[ly - 1][lx] + s_cb[ly + 1][lx], l);
      l = fma(kap, s_cb[ly][lx], l);
      const size_t p = (size_t)gj * nx + gi;
      const TC c = (TC)__ldg(&cn[p]);
      const TC nl = c * fma(c, c, TC(-1));
      m[off + p] = (double)fma(-gl, l, nl);
      cbar[off + p] = (double)s_cb[ly][lx];
    }
  }
}

// NOISE (Cahn-Hilliard-Cook, Sec. 7.7) adds, in pass 2, (2/3) dt eta / k2 with
// eta = sqrt(sigma / (dx dy dt)) div_h rho, the backward-difference divergence
// of the deviates rho (planes rho^x, rho^y of nx*ny per simulation):
// nkx (rho^x_ij - rho^x_{i-1,j}) + nky (rho^y_ij - rho^y_{i,j-1}), nkx and nky
// divided by k2 like the rest of the output.
//   kNoiseRead: caller-given FP64 deviates, read with coalesced row reads and
//     differenced in FP64 into a shared tile.
//   kNoiseDraw: the tile's deviates drawn in place (noise.cuh; even nx, so that
//     a Philox pair never straddles rows): the 16 pairs of each tile row, the
//     pair holding the west halo point, and the row above, with key
//     (seed, sim0 + z) at step *d_step (or `step`), into float tiles; the tile's
//     own deviates are stored to rho as they are drawn.  The divergence of
//     these FP32 values is formed in double-float on the FP32 pipes (exact
//     differences, products with nkx and nky as float pairs, bit-exact float to
//     double conversions): two FP64 additions per point instead of the nine
//     FP64-pipe operations (conversions included) of forming it in FP64.
constexpr int kNoiseNone = 0, kNoiseRead = 1, kNoiseDraw = 2;
// Pass 2's occupancy bound.  Unbounded, its deviate-drawing form takes 54
// registers and 4 blocks per SM: the Cook step measured 0.401 ms against 0.335 ms
// with 6 blocks (40 registers) and 0.339 ms with 8 (same box); the plain step is
// the same 0.2997 ms under all three.
constexpr int kRLapMinBlocks = 6;

template <typename TC, typename TO, int NOISE = kNoiseNone>
__global__ void __launch_bounds__(kT* kRBY, kRLapMinBlocks) ch_rhs_r_kernel(const double* __restrict__ m,
                                                            const double* __restrict__ cn,
                                                            const double* __restrict__ cbar, TO* __restrict__ rT,
                                                            int nx, int ny, int G, TC rho, TC kap, TC kd,
                                                            double* dev = nullptr, double nkx = 0, double nky = 0,
                                                            uint64_t seed = 0, uint64_t sim0 = 0, uint64_t step = 0,
                                                            const uint64_t* __restrict__ d_step = nullptr) {
  __shared__ TC s_m[kT + 2][kT + 3];
  __shared__ TC s_d[kT][kT + 1];
  __shared__ TC s_nz[NOISE == kNoiseRead ? kT : 1][kT + 1];
  // deviate tiles: [a][b] is grid point (i0 - 1 + b, j0 - 1 + a), wrapped; odd pitch for the transposed reads
  __shared__ float s_dx[NOISE == kNoiseDraw ? kT + 1 : 1][kT + 1];
  __shared__ float s_dy[NOISE == kNoiseDraw ? kT + 1 : 1][kT + 1];
  const int z = blockIdx.z;
  const size_t N = (size_t)nx * ny, off = (size_t)z * N;
  m += off;
  cn += off;
  cbar += off;
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int tid = threadIdx.y * kT + threadIdx.x;
  auto stage = [&](int ly, int lx) {
    const int gi = wrap_near(i0 - 1 + lx, nx), gj = wrap_near(j0 - 1 + ly, ny);
    s_m[ly][lx] = (TC)m[(size_t)gj * nx + gi];
  };
#pragma unroll
  for (int k = 0; k < (kT + 2 + kRBY - 1) / kRBY; ++k) {
    const int ly = threadIdx.y + k * kRBY;
    if (ly < kT + 2) stage(ly, threadIdx.x);
  }
  if (tid < 2 * (kT + 2)) stage(tid >> 1, kT + (tid & 1));
#pragma unroll
  for (int k = 0; k < kT / kRBY; ++k) {
    const int lj = threadIdx.y + k * kRBY, li = threadIdx.x;
    const int gi = i0 + li, gj = j0 + lj;
    TC d = 0;
    if (gi < nx && gj < ny) {
      const size_t p = (size_t)gj * nx + gi;
      d = (TC)cbar[p] - (TC)cn[p];  // C^n - C^{n-1}
    }
    s_d[lj][li] = d;
  }
  if constexpr (NOISE == kNoiseRead) {
    const double* rx = dev + (size_t)z * 2 * N;
    const double* ry = rx + N;
#pragma unroll
    for (int k = 0; k < kT / kRBY; ++k) {
      const int lj = threadIdx.y + k * kRBY, li = threadIdx.x;
      const int gi = i0 + li, gj = j0 + lj;
      TC v = 0;
      if (gi < nx && gj < ny) {
        const size_t q = (size_t)gj * nx + gi;
        const size_t qw = (size_t)gj * nx + (gi == 0 ? nx - 1 : gi - 1);
        const size_t qs = (size_t)(gj == 0 ? ny - 1 : gj - 1) * nx + gi;
        v = (TC)fma(nkx, rx[q] - rx[qw], nky * (ry[q] - ry[qs]));
      }
      s_nz[lj][li] = v;
    }
  }
  if constexpr (NOISE == kNoiseDraw) {
    if (d_step) step = *d_step;
    const uint64_t key1 = sim0 + (uint64_t)z;
    double* rx = dev + (size_t)z * 2 * N;
    double* ry = rx + N;
    constexpr int kPairs = kT / 2 + 1;  // per staged row: the west halo's pair, then the tile's
    for (int q = tid; q < (kT + 1) * kPairs; q += kT * kRBY) {
      const int a = q / kPairs, h = q - a * kPairs;
      const int gj = wrap_near(j0 - 1 + a, ny);
      const int gi = h == 0 ? (i0 == 0 ? nx : i0) - 2 : i0 + 2 * (h - 1);  // even: first point of the pair
      if (gi >= nx) continue;                                               // ragged last tile
      float x0, y0, x1, y1;
      const size_t p = (size_t)gj * nx + gi;
      deviate_pair(p >> 1, step, seed, key1, &x0, &y0, &x1, &y1);
      if (h == 0) {
        s_dx[a][0] = x1;
        s_dy[a][0] = y1;
      } else {
        s_dx[a][2 * h - 1] = x0;
        s_dy[a][2 * h - 1] = y0;
        s_dx[a][2 * h] = x1;
        s_dy[a][2 * h] = y1;
        if (a >= 1 && j0 + a - 1 < ny) {  // the tile's own points
          rx[p] = f2d_exact(x0);
          rx[p + 1] = f2d_exact(x1);
          ry[p] = f2d_exact(y0);
          ry[p + 1] = f2d_exact(y1);
        }
      }
    }
  }
  __syncthreads();
  const size_t ldo = (size_t)G * ny;
  ff wx, wy;
  if constexpr (NOISE == kNoiseDraw) {
    wx = d2ff(nkx);
    wy = d2ff(nky);
  }
#pragma unroll
  for (int k = 0; k < kT / kRBY; ++k) {
    const int li = threadIdx.y + k * kRBY, lj = threadIdx.x;  // output (i0 + li, j0 + lj)
    const int ly = lj + 1, lx = li + 1;
    TC l = s_m[ly][lx - 1] + s_m[ly][lx + 1];
    l = fma(rho, s_m[ly - 1][lx] + s_m[ly + 1][lx], l);
    l = fma(kap, s_m[ly][lx], l);
    TC o = fma(-kd, s_d[lj][li], l);
    if constexpr (NOISE == kNoiseRead) o += s_nz[lj][li];
    if constexpr (NOISE == kNoiseDraw) {
      const ff v = ff_add(ff_mul(wx, two_sum(s_dx[lj + 1][li + 1], -s_dx[lj + 1][li])),
                          ff_mul(wy, two_sum(s_dy[lj + 1][li + 1], -s_dy[lj][li + 1])));
      o = (o + f2d_exact(v.hi)) + f2d_exact(v.lo);
    }
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) rT[(size_t)gi * ldo + (size_t)z * ny + gj] = (TO)o;
  }
}

// ---------------------------------------------------------------------------
// Segment-local LU sweeps on interleaved data: element r of segment s of
// system j at [(s*m + r)*ld + j] (+ blockIdx.z * fz for batched y sweeps).
// Writes y = A_seg^{-1} f and the four boundary values (y_0, y_1, y_{m-2},
// y_{m-1}) of every segment (+ blockIdx.z * ybz).  Loads run U rows ahead.
template <typename TIn, typename TC, int U = (sizeof(TC) == 8 ? 8 : 32)>
__global__ void __launch_bounds__(kSolveThreads) spike_local_kernel(const TIn* f, TC* y, int ld, int nsys,
                                                                    DirView<TC> D, TC* __restrict__ yb, size_t fz,
                                                                    size_t ybz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int s = blockIdx.y, m = D.m;
  const int slot = blockIdx.z + j / D.spp;
  const TC a = D.a[slot];
  const TC* lu = D.lu + (size_t)slot * 4 * m;
  f += blockIdx.z * fz;
  y += blockIdx.z * fz;
  yb += blockIdx.z * ybz;
  const size_t L = (size_t)ld;
  const TIn* pf = f + (size_t)s * m * L + j;
  TC* py = y + (size_t)s * m * L + j;
  const TC *ra = lu, *be = lu + m, *ga = lu + 2 * m, *de = lu + 3 * m;
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

// The same sweeps for segments of a multiple of 2U rows (FP64): two prefetch
// buffers used alternately, so there are no per-row bounds tests and no
// register copies between blocks of rows.  Fewer non-FP64 instructions per
// row is what counts here: a single grid gives these sweeps only a few warps
// per SM, and each warp's issue rate bounds how often the FP64 unit is fed.
template <typename TC, int U = 8>
__global__ void __launch_bounds__(kSolveThreads) spike_local_even_kernel(const TC* f, TC* y, int ld, int nsys,
                                                                         DirView<TC> D, TC* __restrict__ yb,
                                                                         size_t fz, size_t ybz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int s = blockIdx.y, m = D.m;
  const int slot = blockIdx.z + j / D.spp;
  const TC a = D.a[slot];
  const TC* lu = D.lu + (size_t)slot * 4 * m;
  f += blockIdx.z * fz;
  y += blockIdx.z * fz;
  yb += blockIdx.z * ybz;
  const size_t L = (size_t)ld;
  const TC* pf = f + (size_t)s * m * L + j;
  TC* py = y + (size_t)s * m * L + j;
  const TC *ra = lu, *be = lu + m, *ga = lu + 2 * m, *de = lu + 3 * m;
  TC g1 = 0, g2 = 0;
  TC b0[U], b1[U];
#pragma unroll
  for (int u = 0; u < U; ++u) b0[u] = pf[(size_t)u * L];
  for (int r0 = 0; r0 < m; r0 += 2 * U) {
#pragma unroll
    for (int u = 0; u < U; ++u) b1[u] = pf[(size_t)(r0 + U + u) * L];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      TC g = fma(-a, g2, b0[u]);
      g = fma(-__ldg(&be[r]), g1, g) * __ldg(&ra[r]);
      py[(size_t)r * L] = g;
      g2 = g1;
      g1 = g;
    }
    if (r0 + 2 * U < m) {
#pragma unroll
      for (int u = 0; u < U; ++u) b0[u] = pf[(size_t)(r0 + 2 * U + u) * L];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + U + u;
      TC g = fma(-a, g2, b1[u]);
      g = fma(-__ldg(&be[r]), g1, g) * __ldg(&ra[r]);
      py[(size_t)r * L] = g;
      g2 = g1;
      g1 = g;
    }
  }
  // back substitution, rows m-1 .. 0
  TC x1 = 0, x2 = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) b0[u] = py[(size_t)(m - 1 - u) * L];
  TC ylast = 0, ylast2 = 0;
  for (int r0 = m - 1; r0 >= 0; r0 -= 2 * U) {
#pragma unroll
    for (int u = 0; u < U; ++u) b1[u] = py[(size_t)(r0 - U - u) * L];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      TC v = fma(-__ldg(&ga[r]), x1, b0[u]);
      v = fma(-__ldg(&de[r]), x2, v);
      py[(size_t)r * L] = v;
      if (u == 0 && r0 == m - 1) ylast = v;
      if (u == 1 && r0 == m - 1) ylast2 = v;
      x2 = x1;
      x1 = v;
    }
    if (r0 - 2 * U >= 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) b0[u] = py[(size_t)(r0 - 2 * U - u) * L];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - U - u;
      TC v = fma(-__ldg(&ga[r]), x1, b1[u]);
      v = fma(-__ldg(&de[r]), x2, v);
      py[(size_t)r * L] = v;
      x2 = x1;
      x1 = v;
    }
  }
  const size_t S = (size_t)nsys;
  yb[(size_t)(4 * s + 0) * S + j] = x1;  // y_0
  yb[(size_t)(4 * s + 1) * S + j] = x2;  // y_1
  yb[(size_t)(4 * s + 2) * S + j] = ylast2;
  yb[(size_t)(4 * s + 3) * S + j] = ylast;
}

// The same reduced solve with R (1, 2 or 4) rows of one segment block per
// thread: each boundary value loaded (from L2) serves R dot products instead of
// one.  Grid (systems / blk, P * 4 / R, Z).  The outputs are multiplied by
// `scale` (the update's k2 for the y sweep).
template <typename TC, int R>
__global__ void __launch_bounds__(kSolveThreads) spike_reducedR_kernel(const TC* __restrict__ yb, DirView<TC> D,
                                                                       TC* __restrict__ tau, int nsys, size_t ybz,
                                                                       TC scale) {
  static_assert(R == 1 || R == 2 || R == 4, "rows per thread");
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const int P = D.P, k = 4 * P;
  const int slot = blockIdx.z + j / D.spp;
  yb += blockIdx.z * ybz;
  tau += blockIdx.z * ybz;
  const int sq = blockIdx.y / (4 / R), q0 = 4 * sq + (blockIdx.y % (4 / R)) * R;  // first output row
  const TC* row = D.rinv + (size_t)slot * k * k + (size_t)q0 * k;
  const int nb = 2 * D.band + 1 < P ? 2 * D.band + 1 : P;
  const int s0 = nb == P ? 0 : sq - D.band;
  TC acc[R];
#pragma unroll
  for (int o = 0; o < R; ++o) acc[o] = 0;
  // block bb + 1's boundary values are loaded while block bb's FMAs issue
  auto col = [&](int bb) {
    const int sb = s0 + bb;
    return 4 * (sb < 0 ? sb + P : (sb >= P ? sb - P : sb));
  };
  int pc = col(0);
  TC v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = yb[(size_t)(pc + u) * nsys + j];
  for (int bb = 0; bb < nb; ++bb) {
    const int pn = bb + 1 < nb ? col(bb + 1) : pc;
    TC nv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) nv[u] = yb[(size_t)(pn + u) * nsys + j];
#pragma unroll
    for (int o = 0; o < R; ++o)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[o] = fma(__ldg(&row[(size_t)o * k + pc + u]), v[u], acc[o]);
    pc = pn;
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = nv[u];
  }
#pragma unroll
  for (int o = 0; o < R; ++o) tau[(size_t)(q0 + o) * nsys + j] = acc[o] * scale;
}

// Spike correction of element (row r of segment s) of system j, applied to y
// as an FMA chain: y - V0 t0 - V1 t1 - W0 b0 - W1 b1 (vw: the slot's spikes).
template <typename TC>
__device__ __forceinline__ TC spike_apply(TC y, const TC* __restrict__ vw, const TC* __restrict__ tau, int m, int P,
                                          int nsys, int s, int r, int j) {
  const int sn = s + 1 == P ? 0 : s + 1, sp = s == 0 ? P - 1 : s - 1;
  const size_t S = (size_t)nsys;
  y = fma(-__ldg(&vw[r]), tau[(size_t)(4 * sn + 0) * S + j], y);
  y = fma(-__ldg(&vw[m + r]), tau[(size_t)(4 * sn + 1) * S + j], y);
  y = fma(-__ldg(&vw[2 * m + r]), tau[(size_t)(4 * sp + 2) * S + j], y);
  return fma(-__ldg(&vw[3 * m + r]), tau[(size_t)(4 * sp + 3) * S + j], y);
}

// x-sweep correction + transpose back: y (element i of row-system (z, j) at
// y[i*(G*ny) + z*ny + j]) -> w[z*nx*ny + j*nx + i].
template <typename TC, typename TO>
__global__ void __launch_bounds__(kT* kBY) ch_xfinish_kernel(const TC* __restrict__ y1, const TC* __restrict__ t1,
                                                             DirView<TC> D, TO* __restrict__ w, int nx, int ny, int G) {
  __shared__ TO s_t[kT][kT + 1];
  const int z = blockIdx.z, m = D.m, P = D.P;
  const TC* vw = D.vw + (size_t)z * 4 * m;
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int j = j0 + threadIdx.x;
  const size_t ld = (size_t)G * ny;
  const int sys = z * ny + j;
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int li = threadIdx.y + k * kBY, i = i0 + li;
    if (i < nx && j < ny) {
      int s, r;
      seg_row(i, m, D.rm, s, r);
      s_t[li][threadIdx.x] = (TO)spike_apply(y1[(size_t)i * ld + sys], vw, t1, m, P, G * ny, s, r, sys);
    }
  }
  __syncthreads();
  w += (size_t)z * nx * ny;
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int lj = threadIdx.y + k * kBY, li = threadIdx.x;
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) w[(size_t)gj * nx + gi] = s_t[li][lj];
  }
}

// y-sweep correction + update C^{n+1} = Cbar + k2 v' for simulation z, where
// v' solves the scaled right-hand side (the reduced values t1 carry k2 already).
// keep_roles = 1 writes C^n into c_prev and C^{n+1} into c_now; otherwise
// C^{n+1} goes into c_prev (the caller swaps the pointers).
template <typename TC>
__global__ void __launch_bounds__(kSolveThreads) ch_update_kernel(const TC* __restrict__ y1, const TC* __restrict__ t1,
                                                                  DirView<TC> D, const double* __restrict__ cbar,
                                                                  double* cn, double* cp, int nx, int ny, double k2,
                                                                  int keep_roles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, z = blockIdx.z, m = D.m, P = D.P;
  if (i >= nx) return;
  const int s = j / m, r = j - s * m;
  const size_t p = (size_t)z * nx * ny + (size_t)j * nx + i;
  t1 += (size_t)z * 4 * P * nx;
  // C^{n+1} = Cbar + k2 y - corr: one FMA, then the four spike terms
  const double nxt = (double)spike_apply((TC)fma(k2, (double)y1[p], cbar[p]), D.vw + (size_t)z * 4 * m, t1, m, P, nx,
                                         s, r, i);
  if (keep_roles) {
    cp[p] = cn[p];
    cn[p] = nxt;
  } else {
    cp[p] = nxt;
  }
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
// Host helpers.
int default_segments(int n, int nsys, int precision) {
  // The dense reduced solve costs 16 P^2 / n operations per point, so P stays
  // near sqrt(n / 8).  FP64 (one thread per segment of every system, streamed
  // from HBM) aims at about 32k independent sweeps and takes fewer segments
  // when there are many systems.  The fused FP32 solves sweep the segments of
  // a block's few systems in shared memory, so their parallelism is x rows (or
  // y columns) per block times P: they keep P near sqrt(n / 8) for any batch.
  int pmax = (int)floor(sqrt(n / 8.0));
  if (pmax < 1) pmax = 1;
  int want = (32768 + nsys - 1) / nsys;
  if (want < 1) want = 1;
  int lim = (pmax < want || precision == CHX_PREC_F32_REFINE) ? pmax : want;
  for (int P = lim; P >= 1; --P)
    if (n % P == 0 && n / P >= 8) return P;
  return 1;
}

// Host FP64 factors of the segment block for one value of a: LU (4m), spikes
// V, W (4m) and the reduced-system inverse ((4P)^2).
int dir_factors_host(int n, int P, double a, std::vector<double>& lu, std::vector<double>& vw,
                     std::vector<double>& rinv) {
  const int m = n / P, k = 4 * P;
  const double b = -4.0 * a, c = 1.0 + 6.0 * a;
  lu.assign(4 * (size_t)m, 0.0);
  vw.assign(4 * (size_t)m, 0.0);
  rinv.assign((size_t)k * k, 0.0);
  std::vector<double> R((size_t)k * k, 0.0);
  double *ra = &lu[0], *be = &lu[m], *ga = &lu[2 * (size_t)m], *de = &lu[3 * (size_t)m];
  int rc = band_factor_host(m, a, b, c, b, a, ra, be, ga, de);
  if (rc) return rc;
  // V = A_seg^{-1} [e at row m-2; d, e at row m-1] (couples t_{s+1}),
  // W = A_seg^{-1} [a, b at row 0; 0, a at row 1] (couples b_{s-1}).
  std::vector<double> rhs(m), col(m);
  for (int q = 0; q < 4; ++q) {
    std::fill(rhs.begin(), rhs.end(), 0.0);
    if (q < 2) {
      rhs[m - 2] += q == 0 ? a : 0.0;  // e = a
      rhs[m - 1] += q == 0 ? b : a;    // d = b, e = a
    } else {
      rhs[0] += q == 2 ? a : b;        // a, b
      rhs[1] += q == 2 ? 0.0 : a;      // 0, a
    }
    band_solve_host(m, a, ra, be, ga, de, rhs.data(), col.data());
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
  return dense_inverse_host(k, R.data(), rinv.data());
}

// Largest circular segment distance whose Rinv block is not below 2^-53 (half
// an FP64 ulp) of the largest block entry.  The blocks decay geometrically with
// the distance (about 3e-4 per segment at the 2048^2 workload's a = 1.9e4, 128
// points per segment), so the first dropped block carries almost all of the
// dropped weight, and it lies below the rounding of the kept terms.
int rinv_band(const std::vector<double>& rinv, int P) {
  const int k = 4 * P;
  std::vector<double> mx(P / 2 + 1, 0.0);
  double all = 0.0;
  for (int q = 0; q < k; ++q)
    for (int p = 0; p < k; ++p) {
      int d = (p / 4 - q / 4 + P) % P;
      if (d > P / 2) d = P - d;
      const double v = fabs(rinv[(size_t)q * k + p]);
      if (v > mx[d]) mx[d] = v;
      if (v > all) all = v;
    }
  int band = 0;
  for (int d = 0; d <= P / 2; ++d)
    if (mx[d] > 0x1p-53 * all) band = d;
  return band;
}

template <typename T>
int dev_alloc(T** p, size_t cnt) {
  if (cudaMalloc(p, cnt * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(CHX_ENOMEM, "ch: allocation of %zu values", cnt);
  }
  return CHX_OK;
}

template <typename T>
int put(T* dst, const std::vector<double>& src) {
  std::vector<T> h(src.size());
  for (size_t i = 0; i < src.size(); ++i) h[i] = (T)src[i];
  return cuda_check(cudaMemcpy(dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "ch: upload");
}

// Uploads v - (float)v for every entry: the low float of the double-float pair
// whose high float put<float> stores.
int put_lo(float* dst, const std::vector<double>& src) {
  std::vector<float> h(src.size());
  for (size_t i = 0; i < src.size(); ++i) h[i] = (float)(src[i] - (double)(float)src[i]);
  return cuda_check(cudaMemcpy(dst, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice), "ch: upload");
}

int dir_alloc(SpikeDir* D, int n, int P, int slots) {
  D->n = n;
  D->P = P;
  D->m = n / P;
  D->slots = slots;
  const size_t m4 = 4 * (size_t)D->m * slots, kk = (size_t)16 * P * P * slots;
  int rc;
  if ((rc = dev_alloc(&D->d_a, slots)) || (rc = dev_alloc(&D->d_lu, m4)) || (rc = dev_alloc(&D->d_vw, m4)) ||
      (rc = dev_alloc(&D->d_rinv, kk)) || (rc = dev_alloc(&D->d_a32, slots)) || (rc = dev_alloc(&D->d_aff, slots)) ||
      (rc = dev_alloc(&D->d_lu4, m4 / 4)) || (rc = dev_alloc(&D->d_vw32, m4)) || (rc = dev_alloc(&D->d_rinv32, kk)) ||
      (rc = dev_alloc(&D->d_vwlo, m4)) || (rc = dev_alloc(&D->d_rinvlo, kk)) || (rc = dev_alloc(&D->d_rb32, kk)) ||
      (rc = dev_alloc(&D->d_rblo, kk)) || (rc = dev_alloc(&D->d_vw4, m4 / 4)) || (rc = dev_alloc(&D->d_vw4lo, m4 / 4)))
    return rc;
  return CHX_OK;
}

// Factorises for `a` and uploads into slot z.
int dir_set(SpikeDir* D, int z, double a) {
  std::vector<double> lu, vw, rinv;
  int rc = dir_factors_host(D->n, D->P, a, lu, vw, rinv);
  if (rc) return rc;
  // the band is shared by the slots: keep the widest any slot has needed
  const int band = rinv_band(rinv, D->P);
  if (band > D->band) D->band = band;
  if (refine_passes(a) > D->passes) D->passes = refine_passes(a);  // likewise the refinement passes
  // rows where the spikes are small enough for a plain FP32 correction: the
  // middle interval where sum_k |vw_k(r)| <= 1, narrowed to what every slot
  // factorised so far allows
  {
    const int m = D->m;
    int lo = 0, hi = m;
    while (lo < m) {
      double t = 0;
      for (int k = 0; k < 4; ++k) t += fabs(vw[(size_t)k * m + lo]);
      if (t <= 1.0) break;
      ++lo;
    }
    while (hi > lo) {
      double t = 0;
      for (int k = 0; k < 4; ++k) t += fabs(vw[(size_t)k * m + hi - 1]);
      if (t <= 1.0) break;
      --hi;
    }
    for (int r = lo; r < hi; ++r) {  // keep the interval contiguous
      double t = 0;
      for (int k = 0; k < 4; ++k) t += fabs(vw[(size_t)k * m + r]);
      if (t > 1.0) { hi = lo; break; }
    }
    if (!D->pset) {
      D->plo = lo;
      D->phi = hi;
      D->pset = true;
    } else {
      D->plo = lo > D->plo ? lo : D->plo;
      D->phi = hi < D->phi ? hi : D->phi;
    }
    if (D->phi < D->plo) D->phi = D->plo;
  }
  const size_t m4 = 4 * (size_t)D->m, kk = (size_t)16 * D->P * D->P;
  const int P = D->P, K = 4 * P;
  std::vector<double> rb(kk);
  for (int d = 0; d < P; ++d)
    for (int u = 0; u < 4; ++u)
      for (int q = 0; q < K; ++q) rb[(size_t)(d * 4 + u) * K + q] = rinv[(size_t)q * K + 4 * ((q / 4 + d) % P) + u];
  const std::vector<double> av(1, a);
  const float2 aff = split_ff(a);
  if ((rc = put(D->d_a + z, av)) || (rc = put(D->d_lu + z * m4, lu)) || (rc = put(D->d_vw + z * m4, vw)) ||
      (rc = put(D->d_rinv + z * kk, rinv)) || (rc = put(D->d_a32 + z, av)) ||
      (rc = put(D->d_vw32 + z * m4, vw)) || (rc = put(D->d_rinv32 + z * kk, rinv)) ||
      (rc = put_lo(D->d_vwlo + z * m4, vw)) || (rc = put_lo(D->d_rinvlo + z * kk, rinv)) ||
      (rc = put(D->d_rb32 + z * kk, rb)) || (rc = put_lo(D->d_rblo + z * kk, rb)))
    return rc;
  {
    const int m = D->m;
    std::vector<double> v4(m4);  // [r][k] = spike k at row r
    for (int r = 0; r < m; ++r)
      for (int k = 0; k < 4; ++k) v4[(size_t)r * 4 + k] = vw[(size_t)k * m + r];
    if ((rc = put((float*)(D->d_vw4 + z * (m4 / 4)), v4)) || (rc = put_lo((float*)(D->d_vw4lo + z * (m4 / 4)), v4)))
      return rc;
    for (int r = 0; r < m; ++r)  // the LU factors the same way: [r][k] = factor k at row r
      for (int k = 0; k < 4; ++k) v4[(size_t)r * 4 + k] = lu[(size_t)k * m + r];
    if ((rc = put((float*)(D->d_lu4 + z * (m4 / 4)), v4))) return rc;
  }
  return cuda_check(cudaMemcpy(D->d_aff + z, &aff, sizeof(float2), cudaMemcpyHostToDevice), "ch: upload");
}

// Copies every slot from slot 0 (device to device).
int dir_replicate(SpikeDir* D) {
  const size_t m4 = 4 * (size_t)D->m, kk = (size_t)16 * D->P * D->P;
  int rc = CHX_OK;
  for (int z = 1; z < D->slots && !rc; ++z) {
    rc = cuda_check(cudaMemcpy(D->d_a + z, D->d_a, sizeof(double), cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_lu + z * m4, D->d_lu, m4 * 8, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_vw + z * m4, D->d_vw, m4 * 8, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_rinv + z * kk, D->d_rinv, kk * 8, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_a32 + z, D->d_a32, 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_aff + z, D->d_aff, 8, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_lu4 + z * (m4 / 4), D->d_lu4, m4 * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_vw32 + z * m4, D->d_vw32, m4 * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_rinv32 + z * kk, D->d_rinv32, kk * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_vwlo + z * m4, D->d_vwlo, m4 * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_rinvlo + z * kk, D->d_rinvlo, kk * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_rb32 + z * kk, D->d_rb32, kk * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_rblo + z * kk, D->d_rblo, kk * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_vw4 + z * (m4 / 4), D->d_vw4, m4 * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
    if (!rc) rc = cuda_check(cudaMemcpy(D->d_vw4lo + z * (m4 / 4), D->d_vw4lo, m4 * 4, cudaMemcpyDeviceToDevice), "ch: replicate");
  }
  return rc;
}

int dir_move(SpikeDir* D, int from, int to, cudaStream_t st) {
  const size_t m4 = 4 * (size_t)D->m, kk = (size_t)16 * D->P * D->P;
  struct { void* base; size_t esz, per; } a[15] = {
      {D->d_a, 8, 1}, {D->d_lu, 8, m4}, {D->d_vw, 8, m4}, {D->d_rinv, 8, kk}, {D->d_a32, 4, 1},
      {D->d_aff, 8, 1}, {D->d_lu4, 4, m4}, {D->d_vw32, 4, m4}, {D->d_rinv32, 4, kk}, {D->d_vwlo, 4, m4},
      {D->d_rinvlo, 4, kk}, {D->d_rb32, 4, kk}, {D->d_rblo, 4, kk}, {D->d_vw4, 4, m4}, {D->d_vw4lo, 4, m4}};
  for (auto& x : a) {
    const size_t b = x.esz * x.per;
    int rc = cuda_check(cudaMemcpyAsync((char*)x.base + to * b, (char*)x.base + from * b, b, cudaMemcpyDeviceToDevice, st),
                        "ch: move parameters");
    if (rc) return rc;
  }
  return CHX_OK;
}

void free_dir(SpikeDir* D) {
  cudaFree(D->d_a); cudaFree(D->d_lu); cudaFree(D->d_vw); cudaFree(D->d_rinv);
  cudaFree(D->d_a32); cudaFree(D->d_aff); cudaFree(D->d_lu4); cudaFree(D->d_vw32); cudaFree(D->d_rinv32);
  cudaFree(D->d_vwlo); cudaFree(D->d_rinvlo); cudaFree(D->d_rb32); cudaFree(D->d_rblo);
  cudaFree(D->d_vw4); cudaFree(D->d_vw4lo);
  *D = SpikeDir();
}

template <typename T>
DirView<T> view(const SpikeDir& D, int spp);
template <>
DirView<double> view<double>(const SpikeDir& D, int spp) {
  return DirView<double>{D.d_a,  D.d_lu,  D.d_vw,  D.d_rinv, D.m,    D.P,   spp,
                         D.band, 1.0f / (float)D.m, nullptr, nullptr,  nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr};
}
template <>
DirView<float> view<float>(const SpikeDir& D, int spp) {
  return DirView<float>{D.d_a32, nullptr, D.d_vw32, D.d_rinv32, D.m,     D.P,    spp,     D.band,
                        1.0f / (float)D.m, D.d_vwlo, D.d_rinvlo, D.d_rb32, D.d_rblo, D.d_vw4, D.d_vw4lo, D.plo, D.phi,
                        D.d_lu4};
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename T>
T* wptr(void* work, size_t off) {
  return (T*)((char*)work + off);
}

}  // namespace

// ---------------------------------------------------------------------------
namespace chx {

FFStep ff_step_params(const ChGroup* g, int G, double* cur, double* prev, void* work, int target, bool balance) {
  FFStep P{};
  P.nx = g->nx;
  P.ny = g->ny;
  P.G = G;
  P.iso = g->kff.rho.x == 1.f && g->kff.rho.y == 0.f;
  P.tx = (int)ceil_div(g->nx, kT);
  P.ty = (int)ceil_div(g->ny, kT);
  P.X = view<float>(g->X, g->ny);
  P.Y = view<float>(g->Y, g->nx);
  P.xs = x_solve_rows(g->nx, g->ny, g->X.P, target);
  y_solve_shape(g->nx, g->ny, G, g->Y.P, target, balance, &P.ysc, &P.ynt, &P.yrb);
  P.xpass = g->X.passes;
  P.ypass = g->Y.passes;
  P.ypad = y_solve_pad(g->Y.m, P.ysc);
  P.lgx = log2_exact(g->X.m);
  P.lgy = log2_exact(g->Y.m);
  P.k = g->kff;
  P.glff = g->d_glff;
  P.noise = g->noise;
  P.nkx = g->nkx;
  P.nky = g->nky;
  P.affX = g->X.d_aff;
  P.affY = g->Y.d_aff;
  P.st[0] = cur;
  P.st[1] = prev;
  P.cur0 = 0;
  P.fhi = wptr<float>(work, g->off_f);
  P.flo = wptr<float>(work, g->off_flo);
  P.whi = wptr<float>(work, g->off_w);
  P.wlo = wptr<float>(work, g->off_wlo);
  P.x0s = wptr<float>(work, g->off_x0);
  P.cbar = wptr<float2>(work, g->off_cb);
  return P;
}


cudaEvent_t Prof::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::release_all() {
  for (auto& e : pend) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto e : pool) cudaEventDestroy(e);
  pend.clear();
  pool.clear();
  slot.clear();
}

int Prof::read(double* ms_out, long long* n_out, int max_slots, int reset) {
  for (size_t k = 0; k < pend.size(); ++k) {
    int rc = cuda_check(cudaEventSynchronize(pend[k].second), "ch_profile_read: event synchronize");
    if (rc) return rc;
    float t = 0.f;
    cudaEventElapsedTime(&t, pend[k].first, pend[k].second);
    ms[slot[k]] += t;
    n[slot[k]] += 1;
    pool.push_back(pend[k].first);
    pool.push_back(pend[k].second);
  }
  pend.clear();
  slot.clear();
  for (int k = 0; k < max_slots && k < kSlots; ++k) {
    if (ms_out) ms_out[k] = ms[k];
    if (n_out) n_out[k] = n[k];
  }
  if (reset)
    for (int k = 0; k < kSlots; ++k) { ms[k] = 0.0; n[k] = 0; }
  return kSlots;
}

ProfScope::ProfScope(Prof* p_, int slot_, cudaStream_t st_) : p(p_), slot(slot_), st(st_) {
  if (p && p->on) {
    e0 = p->get();
    cudaEventRecord(e0, st);
  }
}

ProfScope::~ProfScope() {
  if (e0) {
    cudaEvent_t e1 = p->get();
    cudaEventRecord(e1, st);
    p->pend.push_back({e0, e1});
    p->slot.push_back(slot);
  }
}
#define PROF(slot) ProfScope prof_scope_##slot(prof, slot, st)

std::vector<int> segment_candidates(int n, int nsys, int precision) {
  std::vector<int> out;
  const int d = default_segments(n, nsys, precision);
  out.push_back(d);
  for (int P = 1; P <= n / 8 && P <= 64; ++P)
    if (n % P == 0 && P != d && (P == d / 2 || P == 2 * d || P == d / 4 || P == 4 * d)) out.push_back(P);
  return out;
}

static int group_move_params_gl(ChGroup* g, int from, int to) {
  int rc = cuda_check(cudaMemcpy(g->d_gl + to, g->d_gl + from, 8, cudaMemcpyDeviceToDevice), "ch: replicate");
  if (!rc) rc = cuda_check(cudaMemcpy(g->d_glff + to, g->d_glff + from, 8, cudaMemcpyDeviceToDevice), "ch: replicate");
  return rc;
}

// One-time opt-in of the staged kernels to large dynamic shared memory (kept out
// of launch paths, which may be inside a stream capture).
static int prepare_kernels() {
  static bool done[64] = {false};  // per device
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "ch: cudaGetDevice");
  if (rc || dev < 0 || dev >= 64 || done[dev]) return rc;
  balanced_block(0);  // reads the SM count now, outside any stream capture
  rc = prepare_solve_ff();
  if (!rc) done[dev] = true;
  return rc;
}

int group_init(ChGroup* g, int nx, int ny, double lx, double ly, double gamma, double dt, int precision, int G,
               int px, int py) {
  if (int rc0 = prepare_kernels()) return rc0;
  if (nx < 8 || ny < 8 || nx > 16384 || ny > 16384)
    return fail(CHX_EINVAL, "ch: nx %d, ny %d outside [8, 16384]", nx, ny);
  if (!(lx > 0) || !(ly > 0) || !(dt > 0) || !(gamma >= 0) || !isfinite(lx) || !isfinite(ly) || !isfinite(dt) ||
      !isfinite(gamma))
    return fail(CHX_EINVAL, "ch: lx %g, ly %g, dt %g, gamma %g", lx, ly, dt, gamma);
  if (precision != CHX_PREC_F64 && precision != CHX_PREC_F32_REFINE)
    return fail(CHX_EINVAL, "ch: precision %d", precision);
  if (G < 1 || G > 65535) return fail(CHX_EINVAL, "ch: group size %d", G);
  if ((px && (nx % px || nx / px < 8)) || (py && (ny % py || ny / py < 8)))
    return fail(CHX_EINVAL, "ch: segment counts %d, %d must divide nx, ny with >= 8 points each", px, py);
  g->nx = nx; g->ny = ny; g->G = G; g->precision = precision;
  g->lx = lx; g->ly = ly; g->gamma = gamma; g->dt = dt;
  g->dx = lx / nx; g->dy = ly / ny;
  const double sx = 1.0 / (g->dx * g->dx);
  g->rho = (g->dx * g->dx) / (g->dy * g->dy);
  g->kap = -2.0 * (1.0 + g->rho);
  g->k1 = 2.0 / 3.0;
  g->k2 = (2.0 / 3.0) * dt * sx;
  g->kff.rho = split_ff(g->rho);
  g->kff.kap = split_ff(g->kap);
  g->kff.gl = split_ff(0.0);
  g->kff.k1 = split_ff(g->k1);
  g->kff.k2 = split_ff(g->k2);
  int rc;
  if ((rc = dir_alloc(&g->X, nx, px ? px : default_segments(nx, G * ny, precision), G)) ||
      (rc = dir_alloc(&g->Y, ny, py ? py : default_segments(ny, nx * G, precision), G)) || (rc = dev_alloc(&g->d_gl, G)) ||
      (rc = dev_alloc(&g->d_glff, G)) || (rc = group_set_gamma(g, 0, gamma)) || (rc = dir_replicate(&g->X)) ||
      (rc = dir_replicate(&g->Y))) {
    group_free(g);
    return rc;
  }
  if (precision == CHX_PREC_F32_REFINE && !solve_ff_fits(nx, ny, g->X.P, g->Y.P)) {
    group_free(g);
    return fail(CHX_EUNSUPPORTED, "ch: FP32+refine strips of %d x %d do not fit in shared memory", nx, ny);
  }
  {
    auto dir_bytes = [&](const SpikeDir& D) {
      const size_t m4 = 4 * (size_t)D.m, kk = (size_t)16 * D.P * D.P;
      return (size_t)G * (8 + 4 + 8 + m4 * (8 + 8 + 4 + 4 + 4 + 4 + 4) + kk * (8 + 4 + 4 + 4 + 4));
    };
    g->factor_bytes = dir_bytes(g->X) + dir_bytes(g->Y) + (size_t)G * (sizeof(double) + sizeof(float2));
  }
  for (int z = 1; z < G && !rc; ++z) rc = group_move_params_gl(g, 0, z);
  if (rc) {
    group_free(g);
    return rc;
  }
  const size_t N = (size_t)nx * ny * G;
  const int f64 = precision == CHX_PREC_F64;
  const size_t esz = f64 ? 8 : 4;
  const size_t mix = f64 ? 0 : N * esz;
  size_t off = 0;
  g->off_f = off; off = align256(off + N * esz);
  g->off_flo = off; off = align256(off + mix);
  g->off_w = off; off = align256(off + N * esz);
  g->off_wlo = off; off = align256(off + mix);
  g->off_y1 = off;
  g->off_y2 = off;
  g->off_x0 = off; off = align256(off + mix);  // the fused solves' x0 scratch
  g->off_cb = off; off = align256(off + N * sizeof(double));  // Cbar (FP64, or a double-float pair), formed by the RHS pass
  g->off_m = off; off = align256(off + (f64 ? N * esz : 0));  // M, between the two RHS passes
  // the FP64 step's boundary values and reduced solutions (the fused FP32
  // solves keep theirs in shared memory)
  const size_t kx = f64 ? 4 * (size_t)g->X.P * ny * G : 0, ky = f64 ? 4 * (size_t)g->Y.P * nx * G : 0;
  g->off_ybx = off; off = align256(off + kx * esz);
  g->off_tx = off; off = align256(off + kx * esz);
  g->off_ybx2 = g->off_tx2 = off;
  g->off_yby = off; off = align256(off + ky * esz);
  g->off_ty = off; off = align256(off + ky * esz);
  g->off_yby2 = g->off_ty2 = off;
  g->work_bytes = off;
  return CHX_OK;
}

int group_set_gamma(ChGroup* g, int z, double gamma) {
  if (z < 0 || z >= g->G || !(gamma >= 0) || !isfinite(gamma)) return fail(CHX_EINVAL, "ch: slot %d gamma %g", z, gamma);
  const double ax = (2.0 / 3.0) * gamma * g->dt / (g->dx * g->dx * g->dx * g->dx);
  const double ay = (2.0 / 3.0) * gamma * g->dt / (g->dy * g->dy * g->dy * g->dy);
  int rc;
  if ((rc = dir_set(&g->X, z, ax)) || (rc = dir_set(&g->Y, z, ay))) return rc;
  const double gl = gamma / (g->dx * g->dx);
  const float2 glff = split_ff(gl);
  if ((rc = cuda_check(cudaMemcpy(g->d_gl + z, &gl, sizeof(double), cudaMemcpyHostToDevice), "ch: gamma upload")))
    return rc;
  if (z == 0) g->gamma = gamma;
  return cuda_check(cudaMemcpy(g->d_glff + z, &glff, sizeof(float2), cudaMemcpyHostToDevice), "ch: gamma upload");
}

int group_move_params(ChGroup* g, int from, int to, cudaStream_t st) {
  if (from == to) return CHX_OK;
  int rc;
  if ((rc = dir_move(&g->X, from, to, st)) || (rc = dir_move(&g->Y, from, to, st))) return rc;
  if ((rc = cuda_check(cudaMemcpyAsync(g->d_gl + to, g->d_gl + from, 8, cudaMemcpyDeviceToDevice, st), "ch: move")))
    return rc;
  return cuda_check(cudaMemcpyAsync(g->d_glff + to, g->d_glff + from, 8, cudaMemcpyDeviceToDevice, st), "ch: move");
}

void group_free(ChGroup* g) {
  obs_free(g->obs);
  g->obs = nullptr;
  free_dir(&g->X);
  free_dir(&g->Y);
  cudaFree(g->d_gl);
  cudaFree(g->d_glff);
  g->d_gl = nullptr;
  g->d_glff = nullptr;
}

// Segment-local FP64 sweeps: the register-prefetch kernel (the serial chain
// per system, not load latency, limits these sweeps; a shared-memory staged
// variant measured 82 us against 51 us at 2048^2).
static void launch_local(const double* f, double* y, int ld, int nsys, const DirView<double>& D, double* yb, size_t fz,
                         size_t ybz, int Z, cudaStream_t st) {
  const unsigned blk = balanced_block((size_t)nsys * D.P * Z);
  const dim3 grid(ceil_div(nsys, blk), D.P, Z);
  if (D.m % 16 == 0)
    spike_local_even_kernel<double><<<grid, blk, 0, st>>>(f, y, ld, nsys, D, yb, fz, ybz);
  else
    spike_local_kernel<double, double><<<grid, blk, 0, st>>>(f, y, ld, nsys, D, yb, fz, ybz);
}

// FP64 reduced solves: kReducedRows rows per thread, in single-warp blocks when
// the grid is small (the balance rule of the one-thread-per-system kernels).
// The FP32 path keeps one row per thread: its arithmetic is cheap, and more
// threads hide more load latency (measured 10.4 us against 14 us at 2048^2).
template <typename TC>
static void launch_reduced(const TC* yb, const DirView<TC>& D, TC* tau, int nsys, size_t ybz, int Z, TC scale,
                           cudaStream_t st) {
  const int R = kReducedRows;
  const unsigned blk = balanced_block((size_t)nsys * D.P * (4 / R) * Z);
  spike_reducedR_kernel<TC, kReducedRows><<<dim3(ceil_div(nsys, blk), D.P * (4 / R), Z), blk, 0, st>>>(
      yb, D, tau, nsys, ybz, scale);
}

static void step_f64(ChGroup* g, int G, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st,
                     Prof* prof, int* status) {
  const int nx = g->nx, ny = g->ny;
  const size_t N = (size_t)nx * ny;
  double* f = wptr<double>(work, g->off_f);
  double* w = wptr<double>(work, g->off_w);
  double *ybx = wptr<double>(work, g->off_ybx), *tx = wptr<double>(work, g->off_tx);
  double *yby = wptr<double>(work, g->off_yby), *ty = wptr<double>(work, g->off_ty);
  double* cbar = wptr<double>(work, g->off_cb);
  const dim3 tgrid(ceil_div(nx, kT), ceil_div(ny, kT), G), tblock(kT, kBY), rblock(kT, kRBY);
  const int nsx = G * ny;  // the x sweep: all row systems of the group, interleaved
  const DirView<double> X = view<double>(g->X, ny), Y = view<double>(g->Y, nx);
  const size_t kyz = 4 * (size_t)Y.P * nx;
  double* mf = wptr<double>(work, g->off_m);
  { PROF(kRhs); ch_rhs_m_kernel<double><<<tgrid, rblock, 0, st>>>(cur, prev, mf, cbar, nx, ny, g->rho, g->kap,
                                                                  g->d_gl); }
  {
    PROF(kRhsLap);
    const double kd = g->k1 / g->k2;
    if (g->noise_w)
      ch_rhs_r_kernel<double, double, kNoiseDraw><<<tgrid, rblock, 0, st>>>(
          mf, cur, cbar, f, nx, ny, G, g->rho, g->kap, kd, g->noise_w, g->nkx / g->k2, g->nky / g->k2,
          g->noise_seed, g->noise_sim0, g->noise_step, g->noise_dstep);
    else if (g->noise)
      ch_rhs_r_kernel<double, double, kNoiseRead><<<tgrid, rblock, 0, st>>>(
          mf, cur, cbar, f, nx, ny, G, g->rho, g->kap, kd, const_cast<double*>(g->noise), g->nkx / g->k2,
          g->nky / g->k2);
    else
      ch_rhs_r_kernel<double, double><<<tgrid, rblock, 0, st>>>(mf, cur, cbar, f, nx, ny, G, g->rho, g->kap, kd);
  }
  { PROF(kLocX); launch_local(f, f, nsx, nsx, X, ybx, 0, 0, 1, st); }
  { PROF(kRedX); launch_reduced<double>(ybx, X, tx, nsx, 0, 1, 1.0, st); }
  { PROF(kFinX); ch_xfinish_kernel<double, double><<<tgrid, tblock, 0, st>>>(f, tx, X, w, nx, ny, G); }
  { PROF(kLocY); launch_local(w, w, nx, nx, Y, yby, N, kyz, G, st); }
  { PROF(kRedY); launch_reduced<double>(yby, Y, ty, nx, kyz, G, g->k2, st); }
  { PROF(kUpd); ch_update_kernel<double><<<dim3(ceil_div(nx, kSolveThreads), ny, G), kSolveThreads, 0, st>>>(
        w, ty, Y, cbar, cur, prev, nx, ny, g->k2, keep_roles); }
}

// FP32 + one refinement pass (Sec. 8's float types): the double-float
// right-hand side, then one fused launch per direction (mixed.cu), the last of
// which forms the update.
static void step_f32r(ChGroup* g, int G, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st,
                      Prof* prof) {
  launch_step_ff(ff_step_params(g, G, cur, prev, work, kFFTarget, true), keep_roles, prof, st);
}

int group_cook_deviates(ChGroup* g, int gact, double* rho, uint64_t seed, uint64_t sim0, uint64_t step,
                        const uint64_t* d_step, cudaStream_t st) {
  if (g->precision == CHX_PREC_F64 && g->nx % 2 == 0) {
    g->noise = nullptr;
    g->noise_w = rho;
    g->noise_seed = seed;
    g->noise_sim0 = sim0;
    g->noise_step = step;
    g->noise_dstep = d_step;
    return CHX_OK;
  }
  g->noise = rho;
  g->noise_w = nullptr;
  return launch_noise_normals(rho, g->nx, g->ny, gact, seed, sim0, step, d_step, st);
}

void group_cook_clear(ChGroup* g) {
  g->noise = nullptr;
  g->noise_w = nullptr;
  g->noise_dstep = nullptr;
}

void group_step(ChGroup* g, int gact, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st,
                Prof* prof, int* status) {
  if (g->precision == CHX_PREC_F64) step_f64(g, gact, cur, prev, work, keep_roles, st, prof, status);
  else step_f32r(g, gact, cur, prev, work, keep_roles, st, prof);
}

void ch_plan_free(chx_ch_plan* p) {
  if (!p) return;
  if (p->pair) cudaGraphExecDestroy(p->pair);
  if (p->one) cudaGraphExecDestroy(p->one);
  if (p->cook_pair) cudaGraphExecDestroy(p->cook_pair);
  if (p->d_cook_step) cudaFree(p->d_cook_step);
  if (p->cap) cudaStreamDestroy(p->cap);
  group_free(&p->g);
  if (p->d_partials) cudaFree(p->d_partials);
  if (p->prof) {
    p->prof->release_all();
    delete p->prof;
  }
  hdr_free(&p->hdr);
  p->g.~ChGroup();
  free(p);
}

}  // namespace chx

// ---------------------------------------------------------------------------
extern "C" int ch_plan_create(chx_ch_plan** plan, int nx, int ny, double lx, double ly, double gamma, double dt,
                              int precision) {
  if (!plan) return fail(CHX_EINVAL, "ch_plan_create: null plan pointer");
  *plan = nullptr;
  if (nx < 8 || ny < 8 || nx > 16384 || ny > 16384)
    return fail(CHX_EINVAL, "ch_plan_create: nx %d, ny %d outside [8, 16384]", nx, ny);
  chx_ch_plan* p = (chx_ch_plan*)calloc(1, sizeof(chx_ch_plan));
  if (!p) return fail(CHX_ENOMEM, "ch_plan_create: plan allocation");
  new (&p->g) ChGroup();
  p->prof = new Prof();
  int rc = hdr_init(&p->hdr, kMagicCh);
  if (!rc) rc = group_init(&p->g, nx, ny, lx, ly, gamma, dt, precision, 1);
  if (rc) { ch_plan_free(p); return rc; }
  if (cudaMalloc(&p->d_partials, 3 * (size_t)kDiagBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    p->d_partials = nullptr;
    ch_plan_free(p);
    return fail(CHX_ENOMEM, "ch_plan_create: diagnostics scratch");
  }
  *plan = p;
  return CHX_OK;
}

extern "C" size_t ch_work_bytes(const chx_ch_plan* p) {
  if (!p || p->hdr.magic != kMagicCh) return 0;
  return p->g.work_bytes;
}

extern "C" int ch_step(chx_ch_plan* p, double* c_now, double* c_prev, void* work, int nsteps, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_step: bad plan");
  if (!c_now || !c_prev || !work) return fail(CHX_EINVAL, "ch_step: null pointer");
  if (nsteps < 0) return fail(CHX_EINVAL, "ch_step: nsteps %d < 0", nsteps);
  if (((uintptr_t)work & 255) != 0) return fail(CHX_EINVAL, "ch_step: work must be 256-byte aligned");
  const size_t fb = (size_t)p->g.nx * p->g.ny * sizeof(double);
  const char *a = (const char*)c_now, *b = (const char*)c_prev, *w = (const char*)work;
  const size_t wb = p->g.work_bytes;
  if ((a < b + fb && b < a + fb) || (a < w + wb && w < a + fb) || (b < w + wb && w < b + fb))
    return fail(CHX_EINVAL, "ch_step: c_now, c_prev and work must not overlap");
  cudaStream_t st = (cudaStream_t)stream;
  double *cur = c_now, *prev = c_prev;
  // Graphs replace the per-kernel launches when the call repeats the previous
  // call's pointers (a loop of single steps) or runs four or more steps; a
  // one-off call with new pointers launches eagerly instead of capturing.
  const bool same = p->seen_now == c_now && p->seen_prev == c_prev && p->seen_work == work;
  p->seen_now = c_now;
  p->seen_prev = c_prev;
  p->seen_work = work;
  if (nsteps >= 1 && !p->prof->on && (same || nsteps >= 4)) {
    int rc = CHX_OK;
    if (p->graph_now != c_now || p->graph_prev != c_prev || p->graph_work != work) {
      if (p->pair) cudaGraphExecDestroy(p->pair);
      if (p->one) cudaGraphExecDestroy(p->one);
      p->pair = p->one = nullptr;
      p->graph_now = c_now;
      p->graph_prev = c_prev;
      p->graph_work = work;
    }
    auto capture = [&](cudaGraphExec_t* exec, int two) -> int {
      int r = CHX_OK;
      if (!p->cap) r = cuda_check(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking), "ch_step: stream");
      cudaGraph_t graph = nullptr;
      if (!r) r = cuda_check(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal), "ch_step: capture");
      if (!r) {
        if (two) {
          group_step(&p->g, 1, c_now, c_prev, work, 0, p->cap, nullptr, p->hdr.d_status);
          group_step(&p->g, 1, c_prev, c_now, work, 0, p->cap, nullptr, p->hdr.d_status);
        } else {
          group_step(&p->g, 1, c_now, c_prev, work, 1, p->cap, nullptr, p->hdr.d_status);
        }
        r = cuda_check(cudaStreamEndCapture(p->cap, &graph), "ch_step: end capture");
      }
      if (!r) r = cuda_check(cudaGraphInstantiate(exec, graph, 0), "ch_step: instantiate");
      if (graph) cudaGraphDestroy(graph);
      if (r) *exec = nullptr;
      return r;
    };
    const int pairs = nsteps / 2;
    if (pairs && !p->pair) rc = capture(&p->pair, 1);
    if (!rc && (nsteps & 1) && !p->one) rc = capture(&p->one, 0);
    for (int k = 0; k < pairs && !rc; ++k) rc = cuda_check(cudaGraphLaunch(p->pair, st), "ch_step: graph launch");
    if (!rc && (nsteps & 1)) rc = cuda_check(cudaGraphLaunch(p->one, st), "ch_step: graph launch");
    if (rc) return rc;
    p->hdr.last_stream = st;
    return launch_check("ch_step");
  }
  for (int s = 0; s < nsteps; ++s) {
    const int last = s == nsteps - 1;
    const int keep = last && cur == c_now;
    group_step(&p->g, 1, cur, prev, work, keep, st, p->prof, p->hdr.d_status);
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

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char *x = (const char*)a, *y = (const char*)b;
  return x < y + nb && y < x + na;
}

// Validation shared by the Cahn-Hilliard-Cook entry points; sets the forcing
// weights (2/3) dt sqrt(sigma / (dx dy dt)) / dx and / dy.
static int cook_prepare(chx_ch_plan* p, double* c_now, double* c_prev, void* work, const double* rho, double sigma,
                        const char* name) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "%s: bad plan", name);
  if (!c_now || !c_prev || !work || !rho) return fail(CHX_EINVAL, "%s: null pointer", name);
  if (((uintptr_t)work & 255) != 0) return fail(CHX_EINVAL, "%s: work must be 256-byte aligned", name);
  if (!(sigma >= 0) || !isfinite(sigma)) return fail(CHX_EINVAL, "%s: sigma %g", name, sigma);
  const size_t fb = (size_t)p->g.nx * p->g.ny * sizeof(double), wb = p->g.work_bytes;
  if (overlaps(c_now, fb, c_prev, fb) || overlaps(c_now, fb, work, wb) || overlaps(c_prev, fb, work, wb) ||
      overlaps(rho, 2 * fb, c_now, fb) || overlaps(rho, 2 * fb, c_prev, fb) || overlaps(rho, 2 * fb, work, wb))
    return fail(CHX_EINVAL, "%s: c_now, c_prev, work and rho must not overlap", name);
  const ChGroup& g = p->g;
  const double amp = sqrt(sigma / (g.dx * g.dy * g.dt));
  p->g.nkx = (2.0 / 3.0) * g.dt * amp / g.dx;
  p->g.nky = (2.0 / 3.0) * g.dt * amp / g.dy;
  return CHX_OK;
}

extern "C" int ch_step_noise(chx_ch_plan* p, double* c_now, double* c_prev, void* work, const double* rho,
                             double sigma, void* stream) {
  int rc = cook_prepare(p, c_now, c_prev, work, rho, sigma, "ch_step_noise");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  p->g.noise = rho;
  group_step(&p->g, 1, c_now, c_prev, work, 1, st, p->prof, p->hdr.d_status);
  p->g.noise = nullptr;
  p->hdr.last_stream = st;
  return launch_check("ch_step_noise");
}

extern "C" int ch_cook_run(chx_ch_plan* p, double* c_now, double* c_prev, void* work, double* rho, int nsteps,
                           double sigma, uint64_t seed, uint64_t sim, uint64_t step0, void* stream) {
  int rc = cook_prepare(p, c_now, c_prev, work, rho, sigma, "ch_cook_run");
  if (rc) return rc;
  if (nsteps < 0) return fail(CHX_EINVAL, "ch_cook_run: nsteps %d < 0", nsteps);
  cudaStream_t st = (cudaStream_t)stream;
  int done = 0;
  if (nsteps >= 2 && !p->prof->on) {
    // pairs of forced steps from a captured graph; the deviates' step index
    // lives on the device (set here, advanced inside the graph)
    if (!p->d_cook_step && cudaMalloc(&p->d_cook_step, sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();
      p->d_cook_step = nullptr;
      return fail(CHX_ENOMEM, "ch_cook_run: step counter");
    }
    if (!p->cook_pair || p->cook_now != c_now || p->cook_prev != c_prev || p->cook_work != work ||
        p->cook_rho != rho || p->cook_sigma != sigma || p->cook_seed != seed || p->cook_sim != sim) {
      if (p->cook_pair) cudaGraphExecDestroy(p->cook_pair);
      p->cook_pair = nullptr;
      if (!p->cap) rc = cuda_check(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking), "ch_cook_run: stream");
      cudaGraph_t graph = nullptr;
      if (!rc) rc = cuda_check(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal), "ch_cook_run: capture");
      if (!rc) {
        int crc = CHX_OK;  // launch errors inside the capture; the capture is ended either way
        for (int h = 0; h < 2 && !crc; ++h) {
          crc = group_cook_deviates(&p->g, 1, rho, seed, sim, 0, p->d_cook_step, p->cap);
          if (!crc) {
            group_step(&p->g, 1, h ? c_prev : c_now, h ? c_now : c_prev, work, 0, p->cap, nullptr, p->hdr.d_status);
            crc = launch_step_advance(p->d_cook_step, p->cap);
          }
        }
        group_cook_clear(&p->g);
        rc = cuda_check(cudaStreamEndCapture(p->cap, &graph), "ch_cook_run: end capture");
        if (!rc) rc = crc;
      }
      if (!rc) rc = cuda_check(cudaGraphInstantiate(&p->cook_pair, graph, 0), "ch_cook_run: instantiate");
      if (graph) cudaGraphDestroy(graph);
      if (rc) {
        p->cook_pair = nullptr;
        return rc;
      }
      p->cook_now = c_now;
      p->cook_prev = c_prev;
      p->cook_work = work;
      p->cook_rho = rho;
      p->cook_sigma = sigma;
      p->cook_seed = seed;
      p->cook_sim = sim;
    }
    rc = launch_step_set(p->d_cook_step, step0, st);
    for (int k = 0; k + 2 <= nsteps && !rc; k += 2)
      rc = cuda_check(cudaGraphLaunch(p->cook_pair, st), "ch_cook_run: graph launch");
    if (rc) return rc;
    done = nsteps & ~1;  // pairs leave C^n in c_now
  }
  double *cur = c_now, *prev = c_prev;
  for (int s = done; s < nsteps; ++s) {
    const int keep = s == nsteps - 1 && cur == c_now;
    rc = group_cook_deviates(&p->g, 1, rho, seed, sim, step0 + (uint64_t)s, nullptr, st);
    if (rc) return rc;
    group_step(&p->g, 1, cur, prev, work, keep, st, p->prof, p->hdr.d_status);
    group_cook_clear(&p->g);
    if (!keep) {
      double* t = cur;
      cur = prev;
      prev = t;
    }
    rc = launch_check("ch_cook_run");
    if (rc) return rc;
  }
  p->hdr.last_stream = st;
  return launch_check("ch_cook_run");
}

extern "C" int ch_step_host(chx_ch_plan* p, const double* h_now, const double* h_prev, double* h_out, double* d_now,
                            double* d_prev, void* work, int nsteps, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_step_host: bad plan");
  if (!h_now || !h_prev || !h_out) return fail(CHX_EINVAL, "ch_step_host: null host pointer");
  const size_t fb = (size_t)p->g.nx * p->g.ny * sizeof(double);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = cuda_check(cudaMemcpyAsync(d_now, h_now, fb, cudaMemcpyHostToDevice, st), "ch_step_host: C^n in");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d_prev, h_prev, fb, cudaMemcpyHostToDevice, st), "ch_step_host: C^{n-1} in");
  if (!rc) rc = ch_step(p, d_now, d_prev, work, nsteps, stream);
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h_out, d_now, fb, cudaMemcpyDeviceToHost, st), "ch_step_host: result out");
  p->hdr.last_stream = st;
  return rc;
}

extern "C" int ch_diagnostics(chx_ch_plan* p, const double* c, double* mass_out, double* energy_out, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_diagnostics: bad plan");
  if (!c || !mass_out || !energy_out) return fail(CHX_EINVAL, "ch_diagnostics: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const ChGroup& g = p->g;
  const double hx = 0.5 * g.gamma / (g.dx * g.dx), hy = 0.5 * g.gamma / (g.dy * g.dy);
  ch_diag_partial_kernel<<<kDiagBlocks, kDiagThreads, 0, st>>>(c, g.nx, g.ny, hx, hy, p->d_partials);
  ch_diag_final_kernel<<<1, 32, 0, st>>>(p->d_partials, kDiagBlocks, g.dx * g.dy, mass_out, energy_out,
                                         p->hdr.d_status);
  p->hdr.last_stream = st;
  return launch_check("ch_diagnostics");
}

extern "C" int ch_observables(chx_ch_plan* p, const double* c, double* out, void* stream) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_observables: bad plan");
  if (!c || !out) return fail(CHX_EINVAL, "ch_observables: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = group_observables(&p->g, 1, c, out, 1, p->hdr.d_status, st);
  p->hdr.last_stream = st;
  return rc;
}

extern "C" int ch_profile(chx_ch_plan* p, int enable) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_profile: bad plan");
  p->prof->on = enable ? 1 : 0;
  return CHX_OK;
}

extern "C" int ch_profile_read(chx_ch_plan* p, double* ms, long long* launches, int max_slots, int reset) {
  if (!p || p->hdr.magic != kMagicCh) return fail(CHX_EINVAL, "ch_profile_read: bad plan");
  return p->prof->read(ms, launches, max_slots, reset);
}

extern "C" const char* ch_profile_slot_name(int slot) {
  return (slot >= 0 && slot < kSlots) ? kSlotName[slot] : "";
}
