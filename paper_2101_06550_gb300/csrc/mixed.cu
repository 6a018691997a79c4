// Mixed-precision kernels: FP32 sweeps with one refinement whose residual is
// formed in double-float arithmetic on the FP32 pipes (ff.cuh), for the ADI
// step (CHX_PREC_F32_REFINE) and the batched pentadiagonal solver (refine = 1).
//
// Compiled with --fmad=false: the error-free transformations need every sum
// and product rounded as written; every intended fused multiply-add is an
// explicit fmaf().
//
// Why the residual is not formed with FP64 instructions: on GB300 one FP64
// instruction costs as much issue bandwidth as ~64 FP32 ones, and an FP64
// residual plus the FP64<->FP32 conversions around it would cost as much as the
// FP64 sweeps it is meant to replace.  The double-float residual is accurate to
// ~2^-46 of its terms, which is what one refinement step of an FP32 solve needs.
#include <algorithm>

#include "chgroup.cuh"
#include "ff.cuh"

namespace chx {
namespace {

// right-hand side: 32 x 32 tiles, 32 x 16 threads (three 512-thread blocks per SM)
constexpr int kT = 32, kBY = 16, kSolveThreads = 128;

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

__device__ __forceinline__ ff ffc(float2 c) { return ff{c.x, c.y}; }

// L'(u) = (E + W) + rho (N + S) + kap C at (y, x) of a shared tile stored as
// separate high and low arrays of float2 (one simulation tile per lane); for a
// square cell (rho = 1, kap = -4) the scalings are exact and skipped.  Each
// lane performs the scalar double-float operations in the same order.
template <int LD, bool kIso>
__device__ __forceinline__ ff2 lap_soa(const float2 (*h)[LD], const float2 (*l)[LD], int y, int x, ff2 rho, ff2 kap) {
  ff2 a = ff2_add(ff2{h[y][x - 1], l[y][x - 1]}, ff2{h[y][x + 1], l[y][x + 1]});
  const ff2 b = ff2_add(ff2{h[y - 1][x], l[y - 1][x]}, ff2{h[y + 1][x], l[y + 1][x]});
  const ff2 c{h[y][x], l[y][x]};
  if (kIso) return ff2_add(ff2_add(a, b), ff2_scale2(c, -4.f));
  a = ff2_add(a, ff2_mul(rho, b));
  return ff2_add(a, ff2_mul(kap, c));
}

// Right-hand side of Eq. 3.1 in double-float: r = k2 L'(M) - k1 (C^n - C^{n-1}),
// M = C^3 - C - gl L'(Cbar), in one pass over 32 x 32 tiles (M formed on the
// tile and a 1-point halo ring): whole 32-column rows per warp, r written
// row-major (rhi, rlo: [z][j][i]) for the fused x solve, and Cbar = 2 C^n -
// C^{n-1} as a double-float pair (cbo) for the update.  (The FP64 step
// splits this into two passes to save the ring's FP64 work; here the ring
// costs issue slots on the FP32 pipes.)  A block takes two vertically
// adjacent tiles, A (rows j0 .. j0 + 31) and B (the next 32 rows), one in
// each lane of the packed FP32x2 arithmetic: its shared tiles hold float2
// (lane A, lane B) in separate high and low arrays, so every operand of a
// packed double-float operation is a single 64-bit shared-memory load.
//
// NOISE (Cahn-Hilliard-Cook, Sec. 7.7): the forcing term (2/3) dt eta is
// formed in FP64 on the otherwise idle FP64 unit (one subtraction and one FMA
// per direction) from caller-given or pre-drawn deviates, and added as a
// double-float pair.
template <bool NOISE>
struct RhsSmem {
  float2 cnh[kT + 4][kT + 5], cnl[kT + 4][kT + 5];  // C^n
  float2 cbh[kT + 4][kT + 5], cbl[kT + 4][kT + 5];  // Cbar
  float2 mh[kT + 2][kT + 3], ml[kT + 2][kT + 3];    // M on the tile and its ring
  float2 nzh[NOISE ? kT : 1][kT + 1], nzl[NOISE ? kT : 1][kT + 1];
};

// Tiles (bx, by) and (bx, by + 1) of simulation z, by a 32 x 16 thread block;
// cn / cp are the group's C^n / C^{n-1} buffers.  Tile B may lie past the
// grid's last row: its loads wrap like the halo's and its stores are skipped.
template <bool kIso, bool NOISE>
__device__ __forceinline__ void rhs_ff_pair(RhsSmem<NOISE>& sh, const FFStep& P, const double* __restrict__ cn,
                                            const double* __restrict__ cp, int z, int bx, int by) {
  const int nx = P.nx, ny = P.ny;
  float* __restrict__ rhi = P.fhi;
  float* __restrict__ rlo = P.flo;
  float2* __restrict__ cbo = P.cbar;
  const double* __restrict__ dev = P.noise;
  const double nkx = P.nkx, nky = P.nky;
  const ff2 rho2 = ff2_splat(ffc(P.k.rho)), kap2 = ff2_splat(ffc(P.k.kap)), gl2 = ff2_splat(ffc(P.glff[z]));
  const ff2 k12 = ff2_splat(ffc(P.k.k1)), k22 = ff2_splat(ffc(P.k.k2));
  cn += (size_t)z * nx * ny;
  cp += (size_t)z * nx * ny;
  const int i0 = bx * kT, j0 = by * kT;
  const int tid = threadIdx.y * kT + threadIdx.x;
  // C^n and Cbar = 2 C^n - C^{n-1} at one staged point of both tiles; the four
  // loads are issued before any test of their values
  auto stage = [&](int ly, int lx) {
    const int gi = wrap_near(i0 - 2 + lx, nx);
    const size_t pa = (size_t)wrap_near(j0 - 2 + ly, ny) * nx + gi;
    const size_t pb = (size_t)wrap_near(j0 + kT - 2 + ly, ny) * nx + gi;
    const double xa = cn[pa], ya = cp[pa], xb = cn[pb], yb = cp[pb];
    bool bad = false;
    ff a0 = d2ff_fast(xa, bad), b0 = d2ff_fast(ya, bad), a1 = d2ff_fast(xb, bad), b1 = d2ff_fast(yb, bad);
    if (bad) a0 = d2ff_general(xa), b0 = d2ff_general(ya), a1 = d2ff_general(xb), b1 = d2ff_general(yb);
    const ff2 c = ff2_pack(a0, a1);
    sh.cnh[ly][lx] = c.hi;
    sh.cnl[ly][lx] = c.lo;
    const ff2 cb = ff2_sub(ff2_scale2(c, 2.f), ff2_pack(b0, b1));
    sh.cbh[ly][lx] = cb.hi;
    sh.cbl[ly][lx] = cb.lo;
  };
  for (int ly = threadIdx.y; ly < kT + 4; ly += kBY) stage(ly, threadIdx.x);
  if (tid < 4 * (kT + 4)) stage(tid >> 2, kT + (tid & 3));
  if (NOISE) {
    const size_t N = (size_t)nx * ny;
    const double* rx = dev + (size_t)z * 2 * N;
    const double* ry = rx + N;
    for (int lj = threadIdx.y; lj < kT; lj += kBY) {
      const int li = threadIdx.x, gi = i0 + li;
      ff nzv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gj = j0 + h * kT + lj;
        double v = 0;
        if (gi < nx && gj < ny) {
          const size_t q = (size_t)gj * nx + gi;
          const size_t qw = (size_t)gj * nx + (gi == 0 ? nx - 1 : gi - 1);
          const size_t qs = (size_t)(gj == 0 ? ny - 1 : gj - 1) * nx + gi;
          v = fma(nkx, rx[q] - rx[qw], nky * (ry[q] - ry[qs]));
        }
        nzv[h] = d2ff(v);
      }
      sh.nzh[lj][li] = make_float2(nzv[0].hi, nzv[1].hi);
      sh.nzl[lj][li] = make_float2(nzv[0].lo, nzv[1].lo);
    }
  }
  __syncthreads();
  // M on the tile and its 1-point ring (rows and columns 1 .. 34 of the staged grid)
  auto mstage = [&](int ly, int lx) {
    const ff2 l = lap_soa<kT + 5, kIso>(sh.cbh, sh.cbl, ly, lx, rho2, kap2);
    const ff2 c{sh.cnh[ly][lx], sh.cnl[ly][lx]};
    const ff2 nl = ff2_mul(c, ff2_add_f(ff2_mul(c, c), make_float2(-1.f, -1.f)));
    const ff2 v = ff2_sub(nl, ff2_mul(gl2, l));
    sh.mh[ly - 1][lx - 1] = v.hi;
    sh.ml[ly - 1][lx - 1] = v.lo;
  };
  for (int ly = 1 + threadIdx.y; ly <= kT + 2; ly += kBY) mstage(ly, 1 + threadIdx.x);
  if (tid < 2 * (kT + 2)) mstage(1 + (tid >> 1), kT + 1 + (tid & 1));
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {  // output (i0 + li, j0 + lj) of tile A and the same point of tile B
    const int li = threadIdx.x, lj = threadIdx.y + k * kBY, lx = li + 1;
    const ff2 l = lap_soa<kT + 3, kIso>(sh.mh, sh.ml, lj + 1, lx, rho2, kap2);
    const float2 bh = sh.cbh[lj + 2][lx + 1], bl = sh.cbl[lj + 2][lx + 1];
    const ff2 diff = ff2_sub(ff2{bh, bl}, ff2{sh.cnh[lj + 2][lx + 1], sh.cnl[lj + 2][lx + 1]});  // C^n - C^{n-1}
    ff2 v = ff2_sub(ff2_mul(k22, l), ff2_mul(k12, diff));
    if (NOISE) v = ff2_add(v, ff2{sh.nzh[lj][li], sh.nzl[lj][li]});
    const int gi = i0 + li;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gj = j0 + h * kT + lj;
      if (gi < nx && gj < ny) {
        const size_t q = ((size_t)z * ny + gj) * nx + gi;
        rhi[q] = h ? v.hi.y : v.hi.x;
        rlo[q] = h ? v.lo.y : v.lo.x;
        cbo[q] = h ? make_float2(bh.y, bl.y) : make_float2(bh.x, bl.x);  // Cbar for the update
      }
    }
  }
}

template <bool kIso, bool NOISE>
__global__ void __launch_bounds__(kT* kBY, NOISE ? 2 : 3) ch_rhs_ff_kernel(FFStep P, const double* __restrict__ cn,
                                                            const double* __restrict__ cp) {
  extern __shared__ __align__(16) unsigned char rhs_sm[];
  rhs_ff_pair<kIso, NOISE>(*reinterpret_cast<RhsSmem<NOISE>*>(rhs_sm), P, cn, cp, blockIdx.z, blockIdx.x,
                           2 * blockIdx.y);
}

// x0 = y - (V0 ta + V1 tb + W0 tc + W1 td) for one row of a segment, rounded once
// to float: vh / vl are the row's packed spikes (V0, V1, W0, W1) as high and
// low floats, tt = (ta, tb, tc, td) the next segment's first two reduced
// unknowns and the previous segment's last two.  Near the segment ends the four spike terms are several times
// larger than x0 (|V| up to ~6 at a' = 1.9e4) and cancel, so a plain FP32
// chain would leave several ulps of the terms in x0.  Here every spike is a
// double-float pair (vw + vwlo), the high products are exact (TwoProd), the
// running sum is carried as an unevaluated pair (TwoSum), and only the
// low-part products (~2^-24 of the terms) are rounded in FP32.
__device__ __forceinline__ float corr_exact(float y, float4 vh, float4 vl, float4 tt) {
  const float t[4] = {tt.x, tt.y, tt.z, tt.w};
  const float h[4] = {vh.x, vh.y, vh.z, vh.w};
  const float l[4] = {vl.x, vl.y, vl.z, vl.w};
  float s = y, e = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const ff p = two_prod(h[k], t[k]);
    const ff q = two_sum(s, -p.hi);
    s = q.hi;
    e = e + (q.lo - fmaf(l[k], t[k], p.lo));
  }
  return s + e;
}

// The same for two points that share a row's spikes (two columns of a y strip,
// or two segments of an x row), one per lane: ta and tb their reduced unknowns.
// Each lane performs corr_exact's operations in the same order.
__device__ __forceinline__ float2 corr_exact2(float2 y, float4 vh, float4 vl, float4 ta, float4 tb) {
  const float2 t[4] = {make_float2(ta.x, tb.x), make_float2(ta.y, tb.y), make_float2(ta.z, tb.z),
                       make_float2(ta.w, tb.w)};
  const float h[4] = {vh.x, vh.y, vh.z, vh.w};
  const float l[4] = {vl.x, vl.y, vl.z, vl.w};
  float2 s = y, e = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const ff2 p = two_prod2(make_float2(h[k], h[k]), t[k]);
    const ff2 q = two_sum2(s, f2neg(p.hi));
    s = q.hi;
    e = f2add(e, f2sub(q.lo, __ffma2_rn(make_float2(l[k], l[k]), t[k], p.lo)));
  }
  return f2add(s, e);
}

// Spike sum V0 ta + V1 tb + W0 tc + W1 td of one row for two points (lanes),
// in corr_plain's order.
__device__ __forceinline__ float2 spikes_v2(float4 v, float4 ta, float4 tb) {
  float2 c = __fmul2_rn(make_float2(v.x, v.x), make_float2(ta.x, tb.x));
  c = __ffma2_rn(make_float2(v.y, v.y), make_float2(ta.y, tb.y), c);
  c = __ffma2_rn(make_float2(v.z, v.z), make_float2(ta.z, tb.z), c);
  return __ffma2_rn(make_float2(v.w, v.w), make_float2(ta.w, tb.w), c);
}

// x0 for row r of a segment: the exact form near the segment ends, where the
// spike terms are large and cancel, and the plain FP32 chain in the rows
// [plo, phi) where the spikes' magnitudes sum to at most 1 (there the rounding
// of the terms is no larger than that of x0 itself).
__device__ __forceinline__ float corr_first(float y, const float4* __restrict__ vw4, const float4* __restrict__ vw4lo,
                                            int r, int plo, int phi, float4 t);

// The plain FP32 form, for a row's spikes v already loaded.
__device__ __forceinline__ float corr_plain(float y, float4 v, float4 t) {
  float c = v.x * t.x;
  c = fmaf(v.y, t.y, c);
  c = fmaf(v.z, t.z, c);
  c = fmaf(v.w, t.w, c);
  return y - c;
}

__device__ __forceinline__ float corr_first(float y, const float4* __restrict__ vw4, const float4* __restrict__ vw4lo,
                                            int r, int plo, int phi, float4 t) {
  const float4 v = __ldg(&vw4[r]);
  if (r >= plo && r < phi) return corr_plain(y, v, t);
  return corr_exact(y, v, __ldg(&vw4lo[r]), t);
}

// A x0 for the ADI row (a, -4a, 1 + 6a, -4a, a) at two rows at once (packed
// arithmetic; lane k from w[.].{x,y}): x0 + a * delta^4 x0, the fourth
// difference formed with error-free sums.
__device__ __forceinline__ ff2 adi_apply_ff2(const float2 (&w)[5], ff2 a) {
  const ff2 s2 = two_sum2(w[0], w[4]);
  const ff2 s1 = two_sum2(w[1], w[3]);
  ff2 d = ff2_sub(s2, ff2_scale2(s1, 4.f));
  d = ff2_add(d, two_prod2(make_float2(6.f, 6.f), w[2]));
  return ff2_add_f(ff2_mul(a, d), w[2]);
}

// rho = f - A x0 (high float) for the two rows of a residual pass: f as
// (high, low) floats per row, w[u][d] the five neighbours x0_{e-2..e+2} of row u.
__device__ __forceinline__ float2 resid_pair(const float (&fh)[2], const float (&fl)[2], const float (&w)[2][5],
                                             ff2 a) {
  float2 wv[5];
#pragma unroll
  for (int d = 0; d < 5; ++d) wv[d] = make_float2(w[0][d], w[1][d]);
  return ff2_sub(ff2{make_float2(fh[0], fh[1]), make_float2(fl[0], fl[1])}, adi_apply_ff2(wv, a)).hi;
}

// A w for the ADI row with w itself a double-float pair at each of the five
// points (the second refinement pass, whose iterate is x0 + delta), two
// points per call in the two lanes.
__device__ __forceinline__ ff2 adi_apply_pair2(const ff2 (&w)[5], ff2 a) {
  const ff2 s2 = ff2_add(w[0], w[4]);
  const ff2 s1 = ff2_add(w[1], w[3]);
  ff2 d = ff2_sub(s2, ff2_scale2(s1, 4.f));
  d = ff2_add(d, ff2_mul(ff2{make_float2(6.f, 6.f), make_float2(0.f, 0.f)}, w[2]));
  return ff2_add(w[2], ff2_mul(a, d));
}

// ---------------------------------------------------------------------------
// Batched pentadiagonal refinement (SHARED / UNIFORM coefficients): residual
// r = f - A x0 in double-float (rows of A as double-float constants, f split
// from FP64 by bits), FP32 sweeps for delta, x = x0 + delta added in FP64.
// The forward intermediate is kept as a float in the low half of f's slot.
// Loads of f and x0 run U rows ahead of the sweep.
constexpr int kPU = 8;

__global__ void __launch_bounds__(kSolveThreads) penta_refine_ff_kernel(double* x, const float* __restrict__ x0,
                                                                        int n, int batch,
                                                                        const float* __restrict__ fac,
                                                                        const float2* __restrict__ coef, float s00,
                                                                        float s01, float s10, float s11) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
#define FAC(k, r) __ldg(&fac[(size_t)(k) * m + (r)])
  double* px = x + s;
  const float* p0 = x0 + s;
  // window of x0 at rows r-2..r+2; rows ahead come from the prefetch buffers
  float w0 = p0[(size_t)(n - 2) * B], w1 = p0[(size_t)(n - 1) * B];
  float w2 = p0[0], w3 = p0[B];
  float g1 = 0.f, g2 = 0.f, t0 = 0.f, t1 = 0.f, rt0 = 0.f, rt1 = 0.f;
  double fb[kPU];
  float xb[kPU];  // x0 at rows r+2
#pragma unroll
  for (int u = 0; u < kPU; ++u) {
    fb[u] = (u < n) ? px[(size_t)u * B] : 0.0;
    const int q = u + 2 < n ? u + 2 : u + 2 - n;
    xb[u] = (u < n) ? p0[(size_t)q * B] : 0.f;
  }
  for (int r0 = 0; r0 < n; r0 += kPU) {
    double fn[kPU];
    float xn[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 + kPU + u;
      fn[u] = (r < n) ? px[(size_t)r * B] : 0.0;
      const int q = r + 2 < n ? r + 2 : r + 2 - n;
      xn[u] = (r < n) ? p0[(size_t)q * B] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 + u;
      if (r < n) {
        const float w4 = xb[u];
        const float2 ca = __ldg(&coef[r]), cb = __ldg(&coef[n + r]), cc = __ldg(&coef[2 * n + r]);
        const float2 cd = __ldg(&coef[3 * n + r]), ce = __ldg(&coef[4 * n + r]);
        ff ax = ff_mul_f(ffc(cc), w2);
        ax = ff_add(ax, ff_mul_f(ffc(cb), w1));
        ax = ff_add(ax, ff_mul_f(ffc(cd), w3));
        ax = ff_add(ax, ff_mul_f(ffc(ca), w0));
        ax = ff_add(ax, ff_mul_f(ffc(ce), w4));
        const float res = ff_sub(d2ff(fb[u]), ax).hi;
        if (r < m) {
          float g = fmaf(-FAC(2, r), g2, res);
          g = fmaf(-FAC(1, r), g1, g) * FAC(0, r);
          t0 = fmaf(FAC(5, r), res, t0);
          t1 = fmaf(FAC(6, r), res, t1);
          reinterpret_cast<float*>(px + (size_t)r * B)[0] = g;
          g2 = g1;
          g1 = g;
        } else if (r == m) {
          rt0 = res;
        } else {
          rt1 = res;
        }
        w0 = w1; w1 = w2; w2 = w3; w3 = w4;
      }
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) { fb[u] = fn[u]; xb[u] = xn[u]; }
  }
  const float a0 = rt0 - t0, a1 = rt1 - t1;
  const float xt0 = fmaf(s00, a0, s01 * a1), xt1 = fmaf(s10, a0, s11 * a1);
  px[(size_t)m * B] = f2d_exact(p0[(size_t)m * B]) + f2d_exact(xt0);
  px[(size_t)(m + 1) * B] = f2d_exact(p0[(size_t)(m + 1) * B]) + f2d_exact(xt1);
  float d1 = 0.f, d2 = 0.f;
  float gb[kPU], zb[kPU];
#pragma unroll
  for (int u = 0; u < kPU; ++u) {
    const int r = m - 1 - u;
    gb[u] = (r >= 0) ? reinterpret_cast<const float*>(px + (size_t)r * B)[0] : 0.f;
    zb[u] = (r >= 0) ? p0[(size_t)r * B] : 0.f;
  }
  for (int r0 = m - 1; r0 >= 0; r0 -= kPU) {
    float gn[kPU], zn[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 - kPU - u;
      gn[u] = (r >= 0) ? reinterpret_cast<const float*>(px + (size_t)r * B)[0] : 0.f;
      zn[u] = (r >= 0) ? p0[(size_t)r * B] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        float v = fmaf(-FAC(7, r), xt0, gb[u]);
        v = fmaf(-FAC(8, r), xt1, v);
        v = fmaf(-FAC(3, r), d1, v);
        v = fmaf(-FAC(4, r), d2, v);
        px[(size_t)r * B] = f2d_exact(zb[u]) + f2d_exact(v);
        d2 = d1;
        d1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) { gb[u] = gn[u]; zb[u] = zn[u]; }
  }
#undef FAC
}

// First FP32 solve of the refinement path: reads the FP64 right-hand side by
// its high part (bits, no FP64 instruction), writes x0 (float) into work.
__global__ void __launch_bounds__(kSolveThreads) penta_solve_f32_from_f64_kernel(const double* __restrict__ in,
                                                                                 float* __restrict__ work, int n,
                                                                                 int batch,
                                                                                 const float* __restrict__ fac,
                                                                                 float s00, float s01, float s10,
                                                                                 float s11) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
#define FAC(k, r) __ldg(&fac[(size_t)(k) * m + (r)])
  const double* pin = in + s;
  float* pw = work + s;
  float g1 = 0.f, g2 = 0.f, t0 = 0.f, t1 = 0.f;
  double fb[kPU];
#pragma unroll
  for (int u = 0; u < kPU; ++u) fb[u] = (u < m) ? pin[(size_t)u * B] : 0.0;
  for (int r0 = 0; r0 < m; r0 += kPU) {
    double fn[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 + kPU + u;
      fn[u] = (r < m) ? pin[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const float f = d2ff(fb[u]).hi;
        float g = fmaf(-FAC(2, r), g2, f);
        g = fmaf(-FAC(1, r), g1, g) * FAC(0, r);
        t0 = fmaf(FAC(5, r), f, t0);
        t1 = fmaf(FAC(6, r), f, t1);
        pw[(size_t)r * B] = g;
        g2 = g1;
        g1 = g;
      }
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) fb[u] = fn[u];
  }
  const float r0v = d2ff(pin[(size_t)m * B]).hi - t0, r1v = d2ff(pin[(size_t)(m + 1) * B]).hi - t1;
  const float xt0 = fmaf(s00, r0v, s01 * r1v), xt1 = fmaf(s10, r0v, s11 * r1v);
  pw[(size_t)m * B] = xt0;
  pw[(size_t)(m + 1) * B] = xt1;
  float x1 = 0.f, x2 = 0.f;
  float gb[kPU];
#pragma unroll
  for (int u = 0; u < kPU; ++u) {
    const int r = m - 1 - u;
    gb[u] = (r >= 0) ? pw[(size_t)r * B] : 0.f;
  }
  for (int r0 = m - 1; r0 >= 0; r0 -= kPU) {
    float gn[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 - kPU - u;
      gn[u] = (r >= 0) ? pw[(size_t)r * B] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        float v = fmaf(-FAC(7, r), xt0, gb[u]);
        v = fmaf(-FAC(8, r), xt1, v);
        v = fmaf(-FAC(3, r), x1, v);
        v = fmaf(-FAC(4, r), x2, v);
        pw[(size_t)r * B] = v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) gb[u] = gn[u];
  }
#undef FAC
}

// ---------------------------------------------------------------------------
// Fused FP32 + refinement solves of the ADI step, one launch per direction.
//
// A block owns S whole systems (x: S rows, y: S columns of one simulation) in
// shared memory and runs the refinement of (I + a delta^4) w = f on them:
//   1. FP32 segment sweeps on f_hi (partitioned solve, segments of m rows);
//   2. the reduced (cyclic-coupling) system in double-float;
//   3. x0 = y - spike correction with exact accumulation (corr_exact), to a
//      global scratch x0s (L2-resident: the block rereads it shortly);
//   4. rho = f - A x0 in double-float, back into shared memory;
//   5. FP32 segment sweeps and FP32 reduced system on rho, then the FP32
//      correction: delta;
//   6. w = x0 + delta as an exact double-float pair (x), or the update
//      C^{n+1} = 2 C^n - C^{n-1} + w in FP64 (y).
// Between the phases the data stays on chip; the only global traffic is f,
// the output and the x0 scratch.  Sweep phases use S * P threads (one per
// segment of each system); the others use the whole block.

// In-place sweeps of one segment on shared memory (rows ST apart):
// y = E^{-1} f with the FP32 LU factors of the segment block, f[r] = (ralpha,
// beta, gam, del) of row r (staged in shared memory: one 128-bit load per row,
// at shared-memory rather than L1 latency); boundary values y_0, y_1,
// y_{m-2}, y_{m-1} to yb4.  Rows are taken in blocks of B: the block's values
// and factors are loaded first, so the serial recurrence waits on one load
// latency per block instead of one per row.
template <int ST>
__device__ __forceinline__ void seg_sweep32(float* x, int m, float a, const float4* f, float* yb4, int st = ST) {
  constexpr int B = 8;
  const int STR = ST > 0 ? ST : st;  // ST = 0: the stride st given at run time
  const int mb = m - m % B;
  float g1 = 0.f, g2 = 0.f;
  for (int r0 = 0; r0 < mb; r0 += B) {
    float v[B];
    float4 c[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      v[u] = x[(r0 + u) * STR];
      c[u] = f[r0 + u];
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      float g = fmaf(-a, g2, v[u]);
      g = fmaf(-c[u].y, g1, g) * c[u].x;
      v[u] = g;
      g2 = g1;
      g1 = g;
    }
#pragma unroll
    for (int u = 0; u < B; ++u) x[(r0 + u) * STR] = v[u];
  }
  for (int r = mb; r < m; ++r) {
    const float4 c = f[r];
    float g = fmaf(-a, g2, x[r * STR]);
    g = fmaf(-c.y, g1, g) * c.x;
    x[r * STR] = g;
    g2 = g1;
    g1 = g;
  }
  float x1 = 0.f, x2 = 0.f;
  for (int r = m - 1; r >= mb; --r) {
    const float4 c = f[r];
    float v = fmaf(-c.z, x1, x[r * STR]);
    v = fmaf(-c.w, x2, v);
    x[r * STR] = v;
    x2 = x1;
    x1 = v;
  }
  for (int r0 = mb - B; r0 >= 0; r0 -= B) {
    float v[B];
    float4 c[B];
#pragma unroll
    for (int u = B - 1; u >= 0; --u) {
      v[u] = x[(r0 + u) * STR];
      c[u] = f[r0 + u];
    }
#pragma unroll
    for (int u = B - 1; u >= 0; --u) {
      float t = fmaf(-c[u].z, x1, v[u]);
      t = fmaf(-c[u].w, x2, t);
      v[u] = t;
      x2 = x1;
      x1 = t;
    }
#pragma unroll
    for (int u = 0; u < B; ++u) x[(r0 + u) * STR] = v[u];
  }
  yb4[0] = x1;
  yb4[1] = x2;
  yb4[2] = x[(m - 2) * STR];
  yb4[3] = x[(m - 1) * STR];
}

// Row q of tau = Rinv yb for one system (yb: its 4P boundary values in shared
// memory, 16-byte aligned), with Rinv by block offset (rb, rbl: see
// SpikeDir::d_rb32), over the band's block offsets -band..band (or all P) with
// pointers advanced per block.  FF:
// double-float (exact products, pair-carried sum, one final rounding);
// otherwise plain FP32 FMAs.
template <bool FF, bool SH = false>  // SH: rb / rbl are in shared memory
__device__ __forceinline__ float reduced_row(const float* yb, int q, const float* __restrict__ rb,
                                             const float* __restrict__ rbl, int P, int band) {
  auto ld = [](const float* a) { return SH ? *a : __ldg(a); };
  const int K = 4 * P;
  const int nb = 2 * band + 1 < P ? 2 * band + 1 : P;
  int d = nb == P ? 0 : P - band;  // block offset of the first step (mod P)
  int sb = (q >> 2) + d;
  if (sb >= P) sb -= P;
  const size_t stepw = 4 * (size_t)K;
  const float* rp = rb + d * stepw + q;
  const float* rl = FF ? rbl + d * stepw + q : nullptr;
  float s = 0.f, e = 0.f;
  for (int t = 0; t < nb; ++t) {
    const float4 v = *reinterpret_cast<const float4*>(yb + 4 * sb);
    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (FF) {
        const ff p = two_prod(ld(rp + u * K), vv[u]);
        const ff c = two_sum(s, p.hi);
        s = c.hi;
        e = e + (c.lo + fmaf(ld(rl + u * K), vv[u], p.lo));
      } else {
        s = fmaf(ld(rp + u * K), vv[u], s);
      }
    }
    if (++d == P) {
      d = 0;
      rp -= (P - 1) * stepw;
      if (FF) rl -= (P - 1) * stepw;
    } else {
      rp += stepw;
      if (FF) rl += stepw;
    }
    if (++sb == P) sb = 0;
  }
  return s + e;
}

// Plain FP32 spike correction of one row of a segment: V0 ta + V1 tb + W0 tc + W1 td
// (packed spikes as in corr_exact).
__device__ __forceinline__ float spikes_v(float4 v, float4 t) {
  float c = v.x * t.x;
  c = fmaf(v.y, t.y, c);
  c = fmaf(v.z, t.z, c);
  return fmaf(v.w, t.w, c);
}
__device__ __forceinline__ float spikes32(const float4* __restrict__ vw4, int r, float4 t) {
  return spikes_v(__ldg(&vw4[r]), t);
}

// The reduced unknowns are stored by the segment that uses them: segment p's
// four words are (tau_{4(p+1)}, tau_{4(p+1)+1}, tau_{4(p-1)+2}, tau_{4(p-1)+3})
// (segment indices mod P), the next segment's first two and the previous
// segment's last two, so a row's correction reads them with one 128-bit load.
// Word of reduced unknown q = 4 p + u in that layout:
__device__ __forceinline__ int tau_word(int q, int P) {
  int p = (q >> 2) + ((q & 2) ? 1 : P - 1);
  if (p >= P) p -= P;
  return 4 * p + (q & 3);
}

constexpr int kXThreads = 128;  // x solve: threads per block (rows per block: FFStep::xs)
constexpr int kYThreads = 512;  // y solve: threads per block (columns per block: FFStep::ysc)
constexpr int kYThreadsEns = 256;  // the ensemble's y phase: more, smaller blocks per SM overlap their phases
constexpr int kYUpdRows = 2;       // y update, column pairs: rows whose loads a thread keeps in flight

// Row e of a system -> (segment p, row r in the segment) for segments of m
// rows: shifts when m is a power of two (lg = log2 m), else seg_row.
struct SegMap {
  int m, lg;
  float rm;
  __device__ __forceinline__ void map(int e, int& p, int& r) const {
    if (lg >= 0) {
      p = e >> lg;
      r = e & (m - 1);
    } else {
      seg_row(e, m, rm, p, r);
    }
  }
};

__device__ __forceinline__ int wrap2(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

// x direction.  Rows row0 .. row0 + S - 1 of the group (row = z * ny + j,
// slot z), n = nx points each, row-major f, w and x0s.  Shared memory: the
// rows as [s][segment][m + 1] (the pad makes the segment sweeps of a warp
// bank-conflict free), then the boundary values and reduced solutions.  x0
// goes to the scratch (the residual reads its neighbours there, L2-resident)
// and the residual rho = f - A x0 replaces y in shared memory.  The memory
// phases load a batch of elements before computing on them.  keep_roles: the
// threads the first sweeps leave idle also copy the rows of C^n into the
// C^{n-1} buffer (the kept-roles update then only writes C^{n+1}); the right-
// hand side pass, the last reader of C^{n-1}, has completed.
__device__ __forceinline__ void x_solve_rows(float* sm, const FFStep& PS, int row0, int keep_roles) {
  const float* __restrict__ fhi = PS.fhi;
  const float* __restrict__ flo = PS.flo;
  float* __restrict__ x0s = PS.x0s;
  float* __restrict__ whi = PS.whi;
  float* __restrict__ wlo = PS.wlo;
  const int n = PS.nx, ny = PS.ny, rows = PS.G * PS.ny, lgm = PS.lgx;
  const DirView<float>& D = PS.X;
  const float2* __restrict__ aff = PS.affX;
  const int m = D.m, P = D.P, K = 4 * P, Ls = n + P;
  float* X = sm;
  const int XS = PS.xs;
  float* yb = X + ((XS * Ls + 3) & ~3);  // 16-byte aligned: boundary values by float4
  float* tau = yb + XS * K;
  float4* fs = reinterpret_cast<float4*>(tau + XS * K);  // LU factors of the block's slots
  const SegMap sg{m, lgm, D.rm};
  const int ns = rows - row0 < XS ? rows - row0 : XS;
  const int tid = threadIdx.x;
  const int slot0 = row0 / ny;
  for (int i = tid; i < ((row0 + ns - 1) / ny - slot0 + 1) * m; i += kXThreads) fs[i] = __ldg(&D.lu4[(size_t)slot0 * m + i]);
  for (int s = 0; s < ns; ++s) {
    const float* src = fhi + (size_t)(row0 + s) * n;
    float* xs = X + s * Ls;
    for (int e1 = tid; e1 < n; e1 += 4 * kXThreads) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = e1 + u * kXThreads < n ? src[e1 + u * kXThreads] : 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e1 + u * kXThreads;
        if (e < n) {
          int p, r;
          sg.map(e, p, r);
          xs[e + p] = v[u];
        }
      }
    }
  }
  __syncthreads();
  for (int w = tid; w < ns * P; w += kXThreads) {
    const int s = w / P, p = w - s * P, slot = (row0 + s) / ny;
    seg_sweep32<1>(X + s * Ls + p * (m + 1), m, D.a[slot], fs + (slot - slot0) * m, yb + s * K + 4 * p);
  }
  if (keep_roles) {
    // warps without sweeps copy (all threads, after their sweeps, when every warp has some)
    const int busy = ns * P >= kXThreads - 32 ? 0 : (ns * P + 31) & ~31;
    if (tid >= busy) {
      const double* __restrict__ src = PS.st[PS.cur0] + (size_t)row0 * n;
      double* __restrict__ dst = PS.st[1 - PS.cur0] + (size_t)row0 * n;
      const int len = ns * n, nt = kXThreads - busy;
      constexpr int U = 8;
      for (int i1 = tid - busy; i1 < len; i1 += U * nt) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = i1 + u * nt < len ? src[i1 + u * nt] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (i1 + u * nt < len) dst[i1 + u * nt] = v[u];
      }
    }
  }
  __syncthreads();
  for (int o = tid; o < ns * K; o += kXThreads) {
    const int s = o / K, q = o - s * K, slot = (row0 + s) / ny;
    const size_t ko = (size_t)slot * K * K;
    tau[s * K + tau_word(q, P)] = reduced_row<true>(yb + s * K, q, D.rb + ko, D.rblo + ko, P, D.band);
  }
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    const int slot = (row0 + s) / ny;
    const float4* vw4 = D.vw4 + (size_t)slot * m;
    const float4* vw4l = D.vw4lo + (size_t)slot * m;
    const float* ts = tau + s * K;
    const float* xs = X + s * Ls;
    float* dst = x0s + (size_t)(row0 + s) * n;
    if (kXThreads % m == 0) {
      // m divides the block: the thread's points all sit at row r = tid % m of
      // their segments, so its spikes (and the form of its correction) are fixed
      const int r = tid % m;
      const float4 v = __ldg(&vw4[r]);
      const bool plain = r >= D.plo && r < D.phi;
      const float4 vl = plain ? v : __ldg(&vw4l[r]);
      // points e and e + kXThreads (same row r, segments p and pb) in the two lanes
      for (int e = tid; e < n; e += 2 * kXThreads) {
        const int e2 = e + kXThreads, eb = e2 < n ? e2 : e;
        int p, pb, rr;
        sg.map(e, p, rr);  // rr == r
        sg.map(eb, pb, rr);
        const float4 ta = *reinterpret_cast<const float4*>(ts + 4 * p);
        const float4 tb = *reinterpret_cast<const float4*>(ts + 4 * pb);
        const float2 y = make_float2(xs[e + p], xs[eb + pb]);
        const float2 x0 = plain ? f2sub(y, spikes_v2(v, ta, tb)) : corr_exact2(y, v, vl, ta, tb);
        dst[e] = x0.x;
        if (e2 < n) dst[e2] = x0.y;
      }
      continue;
    }
#pragma unroll 2
    for (int e = tid; e < n; e += kXThreads) {
      int p, r;
      sg.map(e, p, r);
      const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
      dst[e] = corr_first(xs[e + p], vw4, vw4l, r, D.plo, D.phi, t);
    }
  }
  __syncthreads();
  // rho = f - A x0 into shared memory (x0 and its neighbours from the scratch;
  // the periodic wrap only at a row's first and last two points)
  for (int s = 0; s < ns; ++s) {
    const int slot = (row0 + s) / ny;
    const ff2 a = ff2_splat(ffc(aff[slot]));
    const size_t ro = (size_t)(row0 + s) * n;
    const float* x0 = x0s + ro;
    const float* fh0 = fhi + ro;
    const float* fl0 = flo + ro;
    float* xs = X + s * Ls;
    if ((n & 1) == 0 && ((reinterpret_cast<uintptr_t>(fhi) | reinterpret_cast<uintptr_t>(flo) |
                          reinterpret_cast<uintptr_t>(x0s)) & 7) == 0) {
      // a thread takes two adjacent points e, e + 1: f by 8-byte loads and
      // the six values x0_{e-2..e+3} by three (rows start 8-byte aligned)
#pragma unroll 2
      for (int e = 2 * tid; e < n; e += 2 * kXThreads) {
        const float2 fh2 = *reinterpret_cast<const float2*>(fh0 + e);
        const float2 fl2 = *reinterpret_cast<const float2*>(fl0 + e);
        float w[6];
        if (e >= 2 && e + 4 <= n) {
          const float2 a0 = *reinterpret_cast<const float2*>(x0 + e - 2);
          const float2 a1 = *reinterpret_cast<const float2*>(x0 + e);
          const float2 a2 = *reinterpret_cast<const float2*>(x0 + e + 2);
          w[0] = a0.x, w[1] = a0.y, w[2] = a1.x, w[3] = a1.y, w[4] = a2.x, w[5] = a2.y;
        } else {
#pragma unroll
          for (int d = 0; d < 6; ++d) w[d] = x0[wrap2(e + d - 2, n)];
        }
        float2 wv[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) wv[d] = make_float2(w[d], w[d + 1]);
        const float2 rv = ff2_sub(ff2{fh2, fl2}, adi_apply_ff2(wv, a)).hi;
        int p, r;
        sg.map(e, p, r);
        xs[e + p] = rv.x;
        sg.map(e + 1, p, r);
        xs[e + 1 + p] = rv.y;
      }
      continue;
    }
    for (int e1 = tid; e1 < n; e1 += 2 * kXThreads) {
      float fh[2], fl[2], w[2][5];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * kXThreads;
        fh[u] = fl[u] = 0.f;
#pragma unroll
        for (int d = 0; d < 5; ++d) w[u][d] = 0.f;
        if (e < n) {
          fh[u] = fh0[e];
          fl[u] = fl0[e];
          if (e >= 2 && e < n - 2) {
            const float* q = x0 + e;
#pragma unroll
            for (int d = 0; d < 5; ++d) w[u][d] = q[d - 2];
          } else {
#pragma unroll
            for (int d = 0; d < 5; ++d) w[u][d] = x0[wrap2(e + d - 2, n)];
          }
        }
      }
      const float2 rv = resid_pair(fh, fl, w, a);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * kXThreads;
        if (e < n) {
          int p, r;
          sg.map(e, p, r);
          xs[e + p] = u ? rv.y : rv.x;
        }
      }
    }
  }
  __syncthreads();
  for (int w = tid; w < ns * P; w += kXThreads) {
    const int s = w / P, p = w - s * P, slot = (row0 + s) / ny;
    seg_sweep32<1>(X + s * Ls + p * (m + 1), m, D.a[slot], fs + (slot - slot0) * m, yb + s * K + 4 * p);
  }
  __syncthreads();
  for (int o = tid; o < ns * K; o += kXThreads) {
    const int s = o / K, q = o - s * K, slot = (row0 + s) / ny;
    tau[s * K + tau_word(q, P)] = reduced_row<false>(yb + s * K, q, D.rb + (size_t)slot * K * K, nullptr, P, D.band);
  }
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    const int slot = (row0 + s) / ny;
    const float4* vw4 = D.vw4 + (size_t)slot * m;
    const float* ts = tau + s * K;
    const float* xs = X + s * Ls;
    const size_t ro = (size_t)(row0 + s) * n;
    const float* x0 = x0s + ro;
    float* wh = whi + ro;
    float* wl = wlo + ro;
    const bool fixr = kXThreads % m == 0;  // as in the correction: one row of the segment block per thread
    const float4 vr = fixr ? __ldg(&vw4[tid % m]) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e1 = tid; e1 < n; e1 += 4 * kXThreads) {
      float xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = e1 + u * kXThreads < n ? x0[e1 + u * kXThreads] : 0.f;
      float dl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e1 + u * kXThreads;
        dl[u] = 0.f;
        if (e < n) {
          int p, r;
          sg.map(e, p, r);
          const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
          dl[u] = xs[e + p] - (fixr ? spikes_v(vr, t) : spikes32(vw4, r, t));
        }
      }
#pragma unroll
      for (int h = 0; h < 4; h += 2) {  // w = x0 + delta as an exact pair, two rows at once
        const ff2 w = two_sum2(make_float2(xv[h], xv[h + 1]), make_float2(dl[h], dl[h + 1]));
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int e = e1 + (h + k) * kXThreads;
          if (e >= n) break;
          wh[e] = k ? w.hi.y : w.hi.x;
          wl[e] = k ? w.lo.y : w.lo.x;
        }
      }
    }
  }
  // Further refinement passes (stiff operators): rho = f - A w in double-float
  // with the current result w = (whi, wlo) itself a pair (its neighbours from
  // global memory, this block's own rows), delta by the FP32 solve with the
  // coupling in double-float, and w += delta.  Two points per thread per
  // step, e and e + kXThreads.
  for (int pass = 1; pass < PS.xpass; ++pass) {
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      const int slot = (row0 + s) / ny;
      const ff2 a = ff2_splat(ffc(aff[slot]));
      const size_t ro = (size_t)(row0 + s) * n;
      const float* wh0 = whi + ro;
      const float* wl0 = wlo + ro;
      const float* fh0 = fhi + ro;
      const float* fl0 = flo + ro;
      float* xs = X + s * Ls;
      for (int e1 = tid; e1 < n; e1 += 2 * kXThreads) {
        const int e2 = e1 + kXThreads, eb = e2 < n ? e2 : e1;
        ff2 w[5];
  #pragma unroll
        for (int d = 0; d < 5; ++d) {
          const int qa = wrap2(e1 + d - 2, n), qb = wrap2(eb + d - 2, n);
          w[d] = ff2{make_float2(wh0[qa], wh0[qb]), make_float2(wl0[qa], wl0[qb])};
        }
        const ff2 f{make_float2(fh0[e1], fh0[eb]), make_float2(fl0[e1], fl0[eb])};
        const float2 rv = ff2_sub(f, adi_apply_pair2(w, a)).hi;
        int p, r;
        sg.map(e1, p, r);
        xs[e1 + p] = rv.x;
        if (e2 < n) {
          sg.map(e2, p, r);
          xs[e2 + p] = rv.y;
        }
      }
    }
    __syncthreads();
    for (int w = tid; w < ns * P; w += kXThreads) {
      const int s = w / P, p = w - s * P, slot = (row0 + s) / ny;
      seg_sweep32<1>(X + s * Ls + p * (m + 1), m, D.a[slot], fs + (slot - slot0) * m, yb + s * K + 4 * p);
    }
    __syncthreads();
    for (int o = tid; o < ns * K; o += kXThreads) {  // the coupling in double-float, as in the first solve
      const int s = o / K, q = o - s * K, slot = (row0 + s) / ny;
      const size_t ko = (size_t)slot * K * K;
      tau[s * K + tau_word(q, P)] = reduced_row<true>(yb + s * K, q, D.rb + ko, D.rblo + ko, P, D.band);
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      const int slot = (row0 + s) / ny;
      const float4* vw4 = D.vw4 + (size_t)slot * m;
      const float4* vw4l = D.vw4lo + (size_t)slot * m;
      const float* ts = tau + s * K;
      const float* xs = X + s * Ls;
      const size_t ro = (size_t)(row0 + s) * n;
      float* wh = whi + ro;
      float* wl = wlo + ro;
      for (int e = tid; e < n; e += kXThreads) {
        int p, r;
        sg.map(e, p, r);
        const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
        const ff w = ff_add_f(ff{wh[e], wl[e]}, corr_first(xs[e + p], vw4, vw4l, r, D.plo, D.phi, t));
        wh[e] = w.hi;
        wl[e] = w.lo;
      }
    }
  }
}

__global__ void __launch_bounds__(kXThreads, 7) x_solve_ff_kernel(FFStep P, int keep_roles) {
  extern __shared__ __align__(16) float sm[];
  x_solve_rows(sm, P, blockIdx.x * P.xs, keep_roles);
}

// y direction.  Columns col0 .. col0 + S - 1 of simulation z (blockIdx.y),
// n = ny points each; w (the right-hand side), x0s and the fields are
// row-major [z][j][i].  Shared memory: [segment][m rows][S columns] with a
// segment pitch of m S + pad, pad = S - m S (mod 32): the 32 / S segments a
// warp sweeps start S banks apart; then the boundary values and reduced
// solutions (per column at a pitch of 4P + 4 floats).  Thread t handles
// column t % S and rows t / S + k NT / S (NT threads); x0 and the residual as in the x
// solve.  The update C^{n+1} = Cbar + v (v = x0 + delta, an exact pair; Cbar =
// 2 C^n - C^{n-1} as the right-hand side pass's double-float pair) is summed
// in double-float and rounded once to FP64 into cp, or with keep_roles (C^n
// then already copied into cp by the x solve) into cn.
template <int NT>
__device__ __forceinline__ void y_solve_cols(float* sm, const FFStep& PS, double* __restrict__ cn,
                                             double* __restrict__ cp, int keep_roles, int z, int col0) {
  const int nx = PS.nx, n = PS.ny, pad = PS.ypad, lgm = PS.lgy;
  const DirView<float>& D = PS.Y;
  const float2* __restrict__ aff = PS.affY;
  const int S = PS.ysc;      // columns per block (1 to 32)
  const int RR = NT / S;     // rows a pass of the block covers
  const int used = RR * S;   // threads of the row passes (the rest idle there)
  // per-column boundary values and reduced unknowns at a pitch of 4P + 4 floats:
  // 16-byte aligned rows whose starts fall on different banks for a warp's columns
  const int m = D.m, P = D.P, K = 4 * P, K1 = K + 4, pitch = m * S + pad;
  float* X = sm;
  float* yb = X + ((P * pitch + 3) & ~3);
  float* tau = yb + S * K1;
  float4* fs = reinterpret_cast<float4*>(tau + S * K1);  // LU factors of the slot
  const SegMap sg{m, lgm, D.rm};
  const int slot = z;
  const int ns = nx - col0 < S ? nx - col0 : S;
  const size_t zo = (size_t)z * nx * n;
  const int tid = threadIdx.x, s = tid % S, e0 = tid / S;
  const bool live = s < ns && tid < used;
  const int c = col0 + s;
  // column c of the simulation's fields (row e at + e * nx)
  const float* __restrict__ fhi = PS.whi + zo + c;  // the y solve's right-hand side is the x result
  const float* __restrict__ flo = PS.wlo + zo + c;
  float* __restrict__ x0s = PS.x0s + zo + c;
  const float2* __restrict__ cbar = PS.cbar + zo + c;
  // full strips of an even-width grid take the corrections, residual and update
  // two adjacent columns per thread (8- and 16-byte accesses, packed arithmetic)
  double* const dst0 = keep_roles ? cn : cp;  // the update's destination
  const bool pairs = ns == S && S >= 2 && (nx & 1) == 0 &&
                     ((reinterpret_cast<uintptr_t>(PS.whi) | reinterpret_cast<uintptr_t>(PS.wlo) |
                       reinterpret_cast<uintptr_t>(PS.x0s)) & 7) == 0 &&
                     ((reinterpret_cast<uintptr_t>(PS.cbar) | reinterpret_cast<uintptr_t>(dst0)) & 15) == 0;
  double* __restrict__ out2 = dst0 + zo + col0;  // strip base
  // pair passes: column pair cq / 2 of hp, rows rq + k RRp (threads past RRp hp idle there)
  const int hp = S > 1 ? S / 2 : 1, RRp = NT / hp, cq = 2 * (tid % hp), rq = tid / hp;
  const bool plive = tid < RRp * hp;
  cn += zo + c;
  cp += zo + c;
  const size_t ldr = (size_t)RR * nx;  // a pass of the block in elements
  // row e = e0 + k RR of the thread's column is at X[p * pad + tid + k * used]
  // (e S + s = tid + k RR S), p its segment; the global loop pointers
  // advance by a pass of the block
  auto seg = [&](int e) {
    int p, r;
    sg.map(e, p, r);
    return p;
  };
  constexpr int B = 4;  // elements per batch of hoisted global loads
  for (int i = tid; i < m; i += NT) fs[i] = __ldg(&D.lu4[(size_t)slot * m + i]);
  // the slot's reduced inverse by block offset (high, then low floats), when staged
  float* rbs = reinterpret_cast<float*>(fs + m);
  const size_t ko = (size_t)slot * K * K;
  if (PS.yrb) {
    const float4* h4 = reinterpret_cast<const float4*>(D.rb + ko);
    const float4* l4 = reinterpret_cast<const float4*>(D.rblo + ko);
    for (int i = tid; i < K * K / 4; i += NT) {
      reinterpret_cast<float4*>(rbs)[i] = __ldg(&h4[i]);
      reinterpret_cast<float4*>(rbs + K * K)[i] = __ldg(&l4[i]);
    }
  }
  if (live) {
    const float* src = fhi + (size_t)e0 * nx;
    for (int e1 = e0, xi = tid; e1 < n; e1 += B * RR, xi += B * used, src += B * ldr) {
      float v[B];
#pragma unroll
      for (int u = 0; u < B; ++u) v[u] = e1 + u * RR < n ? src[u * ldr] : 0.f;
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (e1 + u * RR < n) X[seg(e1 + u * RR) * pad + xi + u * used] = v[u];
    }
  }
  __syncthreads();
  const float a32 = D.a[slot];
  for (int w = tid; w < S * P; w += NT) {
    const int p = w / S, sw = w - p * S;
    if (sw < ns) seg_sweep32<0>(X + p * pitch + sw, m, a32, fs, yb + sw * K1 + 4 * p, S);
  }
  __syncthreads();
  for (int o = tid; o < S * K; o += NT) {
    const int so = o / K, q = o - so * K;
    if (so < ns)
      tau[so * K1 + tau_word(q, P)] =
          PS.yrb ? reduced_row<true, true>(yb + so * K1, q, rbs, rbs + K * K, P, D.band)
                 : reduced_row<true>(yb + so * K1, q, D.rb + ko, D.rblo + ko, P, D.band);
  }
  __syncthreads();
  const float4* vw4 = D.vw4 + (size_t)slot * m;
  const float4* vw4l = D.vw4lo + (size_t)slot * m;
  const float* ts = tau + s * K1;
  if (pairs) {
    const float* t0 = tau + cq * K1;
    float* __restrict__ x02 = PS.x0s + zo + col0 + cq;
#pragma unroll 2
    for (int e = plive ? rq : n; e < n; e += RRp) {
      int p, r;
      sg.map(e, p, r);
      const float2 yv = *reinterpret_cast<const float2*>(X + p * pad + e * S + cq);
      const float4 ta = *reinterpret_cast<const float4*>(t0 + 4 * p);
      const float4 tb = *reinterpret_cast<const float4*>(t0 + K1 + 4 * p);
      const float4 v = __ldg(&vw4[r]);  // both columns' row r: one spike row, both lanes
      *reinterpret_cast<float2*>(x02 + (size_t)e * nx) =
          r >= D.plo && r < D.phi ? f2sub(yv, spikes_v2(v, ta, tb)) : corr_exact2(yv, v, __ldg(&vw4l[r]), ta, tb);
    }
  } else if (live) {
    float* dst = x0s + (size_t)e0 * nx;
#pragma unroll 2
    for (int e = e0, xi = tid; e < n; e += RR, xi += used, dst += ldr) {
      int p, r;
      sg.map(e, p, r);
      const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
      *dst = corr_first(X[p * pad + xi], vw4, vw4l, r, D.plo, D.phi, t);
    }
  }
  __syncthreads();
  if (pairs) {
    // rho = f - A x0 into shared memory, a thread taking two adjacent columns
    // of a row (8-byte loads of f and of the five x0 neighbours, from the
    // scratch; both lanes of the packed arithmetic) and rows 2 RR apart
    const ff2 a = ff2_splat(ffc(aff[slot]));
    const int RR2 = RRp;
    const size_t cz = zo + col0 + cq;
    const float* __restrict__ fh2 = PS.whi + cz;
    const float* __restrict__ fl2 = PS.wlo + cz;
    const float* __restrict__ x02 = PS.x0s + cz;
    const size_t nx1 = nx;
    for (int e1 = plive ? rq : n; e1 < n; e1 += 2 * RR2) {  // two rows' loads in flight
      float2 h[2], l[2], w[2][5];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * RR2;
        h[u] = l[u] = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < 5; ++d) w[u][d] = make_float2(0.f, 0.f);
        if (e < n) {
          const size_t eo = (size_t)e * nx;
          h[u] = *reinterpret_cast<const float2*>(fh2 + eo);
          l[u] = *reinterpret_cast<const float2*>(fl2 + eo);
          if (e >= 2 && e < n - 2) {
#pragma unroll
            for (int d = 0; d < 5; ++d) w[u][d] = *reinterpret_cast<const float2*>(x02 + eo + (d - 2) * (ptrdiff_t)nx1);
          } else {
#pragma unroll
            for (int d = 0; d < 5; ++d) w[u][d] = *reinterpret_cast<const float2*>(x02 + (size_t)wrap2(e + d - 2, n) * nx);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * RR2;
        if (e < n) *reinterpret_cast<float2*>(X + seg(e) * pad + e * S + cq) = ff2_sub(ff2{h[u], l[u]}, adi_apply_ff2(w[u], a)).hi;
      }
    }
  } else if (live) {  // the same one column per thread (x0 and its neighbours from the scratch)
    const ff2 a = ff2_splat(ffc(aff[slot]));
    const size_t nx1 = nx, nx2 = 2 * (size_t)nx;
    size_t eo1 = (size_t)e0 * nx;
    for (int e1 = e0, xi = tid; e1 < n; e1 += 2 * RR, xi += 2 * used, eo1 += 2 * ldr) {
      float fh[2], fl[2], w[2][5];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * RR;
        fh[u] = fl[u] = 0.f;
#pragma unroll
        for (int d = 0; d < 5; ++d) w[u][d] = 0.f;
        if (e < n) {
          const size_t eo = eo1 + u * ldr;
          fh[u] = fhi[eo];
          fl[u] = flo[eo];
          if (e >= 2 && e < n - 2) {
            const float* q = x0s + eo;
            w[u][0] = q[-(ptrdiff_t)nx2];
            w[u][1] = q[-(ptrdiff_t)nx1];
            w[u][2] = q[0];
            w[u][3] = q[nx1];
            w[u][4] = q[nx2];
          } else {
#pragma unroll
            for (int d = 0; d < 5; ++d) w[u][d] = x0s[(size_t)wrap2(e + d - 2, n) * nx];
          }
        }
      }
      const float2 rv = resid_pair(fh, fl, w, a);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e1 + u * RR;
        if (e < n) X[seg(e) * pad + xi + u * used] = u ? rv.y : rv.x;
      }
    }
  }
  __syncthreads();
  for (int w = tid; w < S * P; w += NT) {
    const int p = w / S, sw = w - p * S;
    if (sw < ns) seg_sweep32<0>(X + p * pitch + sw, m, a32, fs, yb + sw * K1 + 4 * p, S);
  }
  __syncthreads();
  for (int o = tid; o < S * K; o += NT) {
    const int so = o / K, q = o - so * K;
    if (so < ns)
      tau[so * K1 + tau_word(q, P)] = PS.yrb ? reduced_row<false, true>(yb + so * K1, q, rbs, nullptr, P, D.band)
                                             : reduced_row<false>(yb + so * K1, q, D.rb + ko, nullptr, P, D.band);
  }
  __syncthreads();
  if (pairs) {
    const int RR2 = RRp;
    const float* t0 = tau + cq * K1;
    const float* __restrict__ x02 = PS.x0s + zo + col0 + cq;
    const float2* __restrict__ cb2 = PS.cbar + zo + col0 + cq;
    double* __restrict__ o2 = out2 + cq;
    constexpr int UB = kYUpdRows;
    for (int e1 = plive ? rq : n; e1 < n; e1 += UB * RR2) {  // UB rows' loads in flight
      float2 xv[UB];
      float4 cv[UB];  // Cbar of the two columns: (hi, lo, hi, lo)
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e = e1 + u * RR2;
        xv[u] = make_float2(0.f, 0.f);
        cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < n) {
          xv[u] = *reinterpret_cast<const float2*>(x02 + (size_t)e * nx);
          cv[u] = *reinterpret_cast<const float4*>(cb2 + (size_t)e * nx);
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int e = e1 + u * RR2;
        if (e >= n) break;
        int p, r;
        sg.map(e, p, r);
        const float2 dv = *reinterpret_cast<const float2*>(X + p * pad + e * S + cq);
        const float4 ta = *reinterpret_cast<const float4*>(t0 + 4 * p);
        const float4 tb = *reinterpret_cast<const float4*>(t0 + K1 + 4 * p);
        const float2 dl = f2sub(dv, spikes_v2(__ldg(&vw4[r]), ta, tb));
        const ff2 v1 = two_sum2(xv[u], dl);  // x0 + delta as an exact pair
        if (PS.ypass > 1) {  // kept for the further passes
          *reinterpret_cast<float2*>(PS.fhi + zo + col0 + cq + (size_t)e * nx) = v1.hi;
          *reinterpret_cast<float2*>(PS.flo + zo + col0 + cq + (size_t)e * nx) = v1.lo;
          continue;
        }
        const ff2 cb{make_float2(cv[u].x, cv[u].z), make_float2(cv[u].y, cv[u].w)};
        const ff2 v = ff2_add(cb, v1);
        *reinterpret_cast<double2*>(o2 + (size_t)e * nx) = make_double2(ff2d(ff2_first(v)), ff2d(ff2_second(v)));
      }
    }
  } else if (live) {
    size_t eo1 = (size_t)e0 * nx;
    for (int e1 = e0, xi = tid; e1 < n; e1 += B * RR, xi += B * used, eo1 += B * ldr) {
      float xv[B];
      float2 cv[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        xv[u] = 0.f;
        cv[u] = make_float2(0.f, 0.f);
        if (e1 + u * RR < n) {
          xv[u] = x0s[eo1 + u * ldr];
          cv[u] = cbar[eo1 + u * ldr];
        }
      }
      float dl[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int e = e1 + u * RR;
        dl[u] = 0.f;
        if (e < n) {
          int p, r;
          sg.map(e, p, r);
          const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
          dl[u] = X[p * pad + xi + u * used] - spikes32(vw4, r, t);
        }
      }
#pragma unroll
      for (int h = 0; h < B; h += 2) {  // Cbar + (x0 + delta) for two rows at once
        const ff2 cb{make_float2(cv[h].x, cv[h + 1].x), make_float2(cv[h].y, cv[h + 1].y)};
        const ff2 v1 = two_sum2(make_float2(xv[h], xv[h + 1]), make_float2(dl[h], dl[h + 1]));
        const ff2 v = ff2_add(cb, v1);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (e1 + (h + k) * RR >= n) break;
          const size_t q = eo1 + (h + k) * ldr;
          if (PS.ypass > 1) {  // x0 + delta kept for the further passes
            PS.fhi[zo + c + q] = k ? v1.hi.y : v1.hi.x;
            PS.flo[zo + c + q] = k ? v1.lo.y : v1.lo.x;
            continue;
          }
          // kept roles: C^{n+1} over C^n (the x solve has moved C^n into cp)
          (keep_roles ? cn : cp)[q] = ff2d(k ? ff2_second(v) : ff2_first(v));
        }
      }
    }
  }
  // Further refinement passes (stiff operators), one column per thread: rho =
  // f - A v in double-float with v = x0 + delta the pair kept in the right-hand
  // side's buffers (free during the y solve; this block's own columns), delta
  // by the FP32 solve with the coupling in double-float, v += delta, and after
  // the last pass C^{n+1} = Cbar + v.
  float* __restrict__ vh = PS.fhi + zo + c;
  float* __restrict__ vl = PS.flo + zo + c;
  for (int pass = 1; pass < PS.ypass; ++pass) {
    const bool last = pass + 1 == PS.ypass;
    __syncthreads();
    if (live) {
      const ff2 a = ff2_splat(ffc(aff[slot]));
      for (int e1 = e0, xi = tid; e1 < n; e1 += 2 * RR, xi += 2 * used) {
        const int e2 = e1 + RR, eb = e2 < n ? e2 : e1;
        ff2 w[5];
  #pragma unroll
        for (int d = 0; d < 5; ++d) {
          const size_t qa = (size_t)wrap2(e1 + d - 2, n) * nx, qb = (size_t)wrap2(eb + d - 2, n) * nx;
          w[d] = ff2{make_float2(vh[qa], vh[qb]), make_float2(vl[qa], vl[qb])};
        }
        const size_t fa = (size_t)e1 * nx, fb = (size_t)eb * nx;
        const ff2 f{make_float2(fhi[fa], fhi[fb]), make_float2(flo[fa], flo[fb])};
        const float2 rv = ff2_sub(f, adi_apply_pair2(w, a)).hi;
        X[seg(e1) * pad + xi] = rv.x;
        if (e2 < n) X[seg(e2) * pad + xi + used] = rv.y;
      }
    }
    __syncthreads();
    for (int w = tid; w < S * P; w += NT) {
      const int p = w / S, sw = w - p * S;
      if (sw < ns) seg_sweep32<0>(X + p * pitch + sw, m, a32, fs, yb + sw * K1 + 4 * p, S);
    }
    __syncthreads();
    for (int o = tid; o < S * K; o += NT) {  // the coupling in double-float, as in the first solve
      const int so = o / K, q = o - so * K;
      if (so < ns)
        tau[so * K1 + tau_word(q, P)] =
            PS.yrb ? reduced_row<true, true>(yb + so * K1, q, rbs, rbs + K * K, P, D.band)
                   : reduced_row<true>(yb + so * K1, q, D.rb + ko, D.rblo + ko, P, D.band);
    }
    __syncthreads();
    if (live) {
      double* __restrict__ dst = keep_roles ? cn : cp;  // this thread's column
      for (int e = e0, xi = tid; e < n; e += RR, xi += used) {
        int p, r;
        sg.map(e, p, r);
        const float4 t = *reinterpret_cast<const float4*>(ts + 4 * p);
        const size_t q = (size_t)e * nx;
        const ff v = ff_add_f(ff{vh[q], vl[q]}, corr_first(X[p * pad + xi], vw4, vw4l, r, D.plo, D.phi, t));
        if (!last) {
          vh[q] = v.hi;
          vl[q] = v.lo;
          continue;
        }
        const float2 cb = cbar[q];
        dst[q] = ff2d(ff_add(ff{cb.x, cb.y}, v));
      }
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : 2) y_solve_ff_kernel(FFStep P, double* cn, double* cp,
                                                                            int keep_roles) {
  extern __shared__ __align__(16) float sm[];
  y_solve_cols<NT>(sm, P, cn, cp, keep_roles, blockIdx.y, blockIdx.x * P.ysc);
}

// ---------------------------------------------------------------------------
// Ensemble phase kernels: block b takes items b, b + gridDim.x, ... of the
// packed order (every group's items, group after group); see chgroup.cuh.
// The group of a block's current item, with that group's step parameters
// cached in shared memory.  A block's items increase, so its group only moves
// forward; the parameters are copied (by all threads, then a barrier) when the
// group changes, and the item numbers the group covers are kept in registers,
// so an item of the same group starts with no global-memory round trip.  Every
// thread of the block makes the same calls; the caller's barrier at the end of
// each item keeps the copy from overwriting parameters still in use.
struct EnsCursor {
  int k = -1, first = 0, end = 0;
  __device__ __forceinline__ const FFStep& at(FFStep& sP, const FFStep* __restrict__ steps,
                                              const int* __restrict__ order, const int* __restrict__ start, int ng,
                                              int it) {
    if (it >= end) {
      int kn = k + 1;
      while (kn + 1 < ng && start[kn + 1] <= it) ++kn;
      k = kn;
      first = start[kn];
      end = start[kn + 1];
      const int* src = reinterpret_cast<const int*>(steps + order[kn]);
      int* dst = reinterpret_cast<int*>(&sP);
      const int nt = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
      for (int w = t; w < (int)(sizeof(FFStep) / sizeof(int)); w += nt) dst[w] = src[w];
      __syncthreads();
    }
    return sP;
  }
};

// An item is a pair of vertically adjacent tiles (rhs_ff_pair).
template <bool NOISE>
__global__ void __launch_bounds__(kT* kBY, NOISE ? 2 : 3) ens_rhs_ff_kernel(const FFStep* __restrict__ steps,
                                                          const int* __restrict__ order,
                                                          const int* __restrict__ start, int ng, int nitems,
                                                          int parity) {
  extern __shared__ __align__(16) unsigned char rhs_sm[];
  __shared__ FFStep sP;
  EnsCursor cur;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const FFStep& P = cur.at(sP, steps, order, start, ng, it);
    const int typ = (P.ty + 1) / 2, idx = it - cur.first, tpz = P.tx * typ;
    const int z = idx / tpz, rem = idx - z * tpz, byp = rem / P.tx, bx = rem - byp * P.tx, by = 2 * byp;
    const int c = P.cur0 ^ parity;
    if (NOISE && P.noise) {
      auto& sh = *reinterpret_cast<RhsSmem<NOISE>*>(rhs_sm);
      if (P.iso) rhs_ff_pair<true, NOISE>(sh, P, P.st[c], P.st[1 - c], z, bx, by);
      else rhs_ff_pair<false, NOISE>(sh, P, P.st[c], P.st[1 - c], z, bx, by);
    } else {
      // tiles without forcing: the NOISE branch of the tile is compiled out
      auto& sh = *reinterpret_cast<RhsSmem<false>*>(rhs_sm);
      if (P.iso) rhs_ff_pair<true, false>(sh, P, P.st[c], P.st[1 - c], z, bx, by);
      else rhs_ff_pair<false, false>(sh, P, P.st[c], P.st[1 - c], z, bx, by);
    }
    __syncthreads();  // the next item reuses the shared tiles and parameters
  }
}

__global__ void __launch_bounds__(kXThreads, 7) ens_x_ff_kernel(const FFStep* __restrict__ steps,
                                                                const int* __restrict__ order,
                                                                const int* __restrict__ start, int ng, int nitems) {
  extern __shared__ __align__(16) float sm[];
  __shared__ FFStep sP;
  EnsCursor cur;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const FFStep& P = cur.at(sP, steps, order, start, ng, it);
    x_solve_rows(sm, P, (it - cur.first) * P.xs, 0);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kYThreadsEns, 4) ens_y_ff_kernel(const FFStep* __restrict__ steps,
                                                                const int* __restrict__ order,
                                                                const int* __restrict__ start, int ng, int nitems,
                                                                int parity) {
  extern __shared__ __align__(16) float sm[];
  __shared__ FFStep sP;
  EnsCursor cur;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const FFStep& P = cur.at(sP, steps, order, start, ng, it);
    const int idx = it - cur.first, nstrip = (P.nx + P.ysc - 1) / P.ysc;
    const int z = idx / nstrip, col0 = (idx - z * nstrip) * P.ysc, c = P.cur0 ^ parity;
    y_solve_cols<kYThreadsEns>(sm, P, P.st[c], P.st[1 - c], 0, z, col0);
    __syncthreads();
  }
}

}  // namespace

void launch_penta_refine_ff(double* x, float* work, int n, int batch, const float* fac32, const float2* coef_ff,
                            const float* s32, cudaStream_t st) {
  const unsigned blk = balanced_block(batch), grid = ceil_div(batch, blk);
  penta_solve_f32_from_f64_kernel<<<grid, blk, 0, st>>>(x, work, n, batch, fac32, s32[0], s32[1], s32[2],
                                                                   s32[3]);
  penta_refine_ff_kernel<<<grid, blk, 0, st>>>(x, work, n, batch, fac32, coef_ff, s32[0], s32[1], s32[2],
                                                         s32[3]);
}


// ---------------------------------------------------------------------------
// Fused solves: shared-memory sizes, column counts and launches.
size_t x_solve_smem(int n, int ny, int P, int xs) {
  const int slots = std::min(xs, (xs - 1 + ny - 1) / ny + 1);  // most slots xs consecutive rows can touch
  return sizeof(float) * ((((size_t)xs * (n + P) + 3) & ~(size_t)3) + 2 * (size_t)xs * 4 * P + 4 * (size_t)(n / P) * slots);
}
int y_solve_pad(int m, int S) { return (((S - m * S) % 32) + 32) % 32; }
size_t y_solve_smem(int n, int P, int S, int rbs) {
  const int m = n / P;
  return sizeof(float) * ((((size_t)P * (m * S + y_solve_pad(m, S)) + 3) & ~(size_t)3) + 2 * (size_t)S * (4 * P + 4) +
                          4 * (size_t)m + (rbs ? 2 * (size_t)16 * P * P : 0));
}
int log2_exact(int m) {
  int lg = 0;
  while ((1 << lg) < m) ++lg;
  return (1 << lg) == m ? lg : -1;
}
namespace {
constexpr size_t kSmemMax = 227 * 1024;
}  // namespace

// Tile shapes of the fused solves: about `target` points per block (so that a
// block's phases amortise their barriers on small grids), as a power of two;
// the y solve takes at least 8 columns (32-byte row segments) and at most 32,
// the x solve at most 32 rows; both shrink until two blocks fit on an SM (or,
// failing that, one).  0: nothing fits.
static int pow2_floor(int v) {
  int p = 1;
  while (2 * p <= v) p *= 2;
  return p;
}
int x_solve_rows(int n, int ny, int P, int target) {
  int xs = pow2_floor(std::min(32, std::max(2, target / n)));
  while (xs > 1 && x_solve_smem(n, ny, P, xs) > 100 * 1024) xs /= 2;
  return x_solve_smem(n, ny, P, xs) <= kSmemMax ? xs : 0;
}
int y_solve_cols(int n, int P, int target) {
  int S = pow2_floor(std::min(32, std::max(8, target / n)));
  while (S > 1 && y_solve_smem(n, P, S) > 100 * 1024) S /= 2;
  return y_solve_smem(n, P, S) <= kSmemMax ? S : 0;
}

void y_solve_shape(int nx, int ny, int G, int P, int target, bool balance, int* S_out, int* nt_out, int* rbs_out) {
  const int S0 = y_solve_cols(ny, P, target);
  *S_out = S0;
  *nt_out = 512;
  *rbs_out = 0;
  if (!balance || S0 < 1) return;
  // stage the reduced inverse when it keeps the blocks per SM (two of 512 threads, or one of 1024)
  struct Pick {
    static void rbs(int ny_, int P_, int S_, int nt_, int* out) {
      const size_t with = y_solve_smem(ny_, P_, S_, 1);
      *out = nt_ == 512 ? with <= 112 * 1024 : with <= kSmemMax - 1024;
    }
  };
  Pick::rbs(ny, P, S0, 512, rbs_out);
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
    cudaGetLastError();
    if (sms < 1) return;
  }
  // columns on the busiest SM: strips are handed out one per SM in turn
  auto cost = [&](int S) { return (long long)ceil_div((size_t)ceil_div((size_t)nx, (size_t)S) * G, (size_t)sms) * S; };
  long long best = cost(S0);
  for (int S = 4; S <= 32; S += 2) {
    const size_t sm = y_solve_smem(ny, P, S);
    if (sm > kSmemMax - 1024) continue;
    const long long c = cost(S);
    if (c * 20 < best * 19) {  // at least 5% fewer columns on the busiest SM
      best = c;
      *S_out = S;
      *nt_out = sm <= 112 * 1024 ? 512 : 1024;  // two 512-thread blocks per SM, else one of 1024
      Pick::rbs(ny, P, S, *nt_out, rbs_out);
    }
  }
}

static_assert(sizeof(FFStep) <= 1024, "the ensemble kernels' static parameter copy must fit the reserved kilobyte");
size_t ens_phase_smem_max() { return kSmemMax - 1024; }

int prepare_solve_ff() {
  int rc = cuda_check(cudaFuncSetAttribute(x_solve_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax),
                      "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(y_solve_ff_kernel<kYThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(y_solve_ff_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax), "mixed: shared-memory opt-in");
  // the right-hand side's shared tiles (two tiles, high and low arrays) exceed the 48 KB default
  const int r1 = (int)sizeof(RhsSmem<true>), r0 = (int)sizeof(RhsSmem<false>);
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ch_rhs_ff_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, r1), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ch_rhs_ff_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, r1), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ch_rhs_ff_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, r0), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ch_rhs_ff_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, r0), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ens_rhs_ff_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, r1), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ens_rhs_ff_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, r0), "mixed: shared-memory opt-in");
  // the ensemble kernels also hold a group's parameters in static shared memory
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ens_x_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ens_phase_smem_max()), "mixed: shared-memory opt-in");
  if (!rc) rc = cuda_check(cudaFuncSetAttribute(ens_y_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ens_phase_smem_max()), "mixed: shared-memory opt-in");
  return rc;
}

bool solve_ff_fits(int nx, int ny, int px, int py) {
  return x_solve_rows(nx, ny, px, kFFTarget) > 0 && y_solve_cols(ny, py, kFFTarget) > 0;
}

void launch_step_ff(const FFStep& P, int keep_roles, Prof* prof, cudaStream_t st) {
  {
    ProfScope ps(prof, kRhs, st);
    const dim3 grid(P.tx, (P.ty + 1) / 2, P.G), block(kT, kBY);  // a block per pair of tiles
    const size_t s1 = sizeof(RhsSmem<true>), s0 = sizeof(RhsSmem<false>);
    if (P.noise && P.iso) ch_rhs_ff_kernel<true, true><<<grid, block, s1, st>>>(P, P.st[0], P.st[1]);
    else if (P.noise) ch_rhs_ff_kernel<false, true><<<grid, block, s1, st>>>(P, P.st[0], P.st[1]);
    else if (P.iso) ch_rhs_ff_kernel<true, false><<<grid, block, s0, st>>>(P, P.st[0], P.st[1]);
    else ch_rhs_ff_kernel<false, false><<<grid, block, s0, st>>>(P, P.st[0], P.st[1]);
  }
  {
    ProfScope ps(prof, kXSolve, st);
    x_solve_ff_kernel<<<ceil_div((size_t)P.G * P.ny, P.xs), kXThreads, x_solve_smem(P.nx, P.ny, P.X.P, P.xs), st>>>(P, keep_roles);
  }
  {
    ProfScope ps(prof, kYSolve, st);
    const dim3 grid(ceil_div(P.nx, P.ysc), P.G);
    const size_t smem = y_solve_smem(P.ny, P.Y.P, P.ysc, P.yrb);
    if (P.ynt == 1024) y_solve_ff_kernel<1024><<<grid, 1024, smem, st>>>(P, P.st[0], P.st[1], keep_roles);
    else y_solve_ff_kernel<kYThreads><<<grid, kYThreads, smem, st>>>(P, P.st[0], P.st[1], keep_roles);
  }
}

int ens_phase_items(int phase, const FFStep& P) {
  if (phase == 0) return P.tx * ((P.ty + 1) / 2) * P.G;  // pairs of tiles
  if (phase == 1) return (int)ceil_div((size_t)P.G * P.ny, P.xs);
  return (int)ceil_div(P.nx, P.ysc) * P.G;
}

int ens_phase_occupancy(int phase, size_t smem) {
  int b = 0;
  if (phase == 0) {  // smem: whether the launch is the Cook-forcing variant
    if (smem) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_rhs_ff_kernel<true>, kT * kBY, sizeof(RhsSmem<true>));
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_rhs_ff_kernel<false>, kT * kBY, sizeof(RhsSmem<false>));
  }
  else if (phase == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_x_ff_kernel, kXThreads, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_y_ff_kernel, kYThreadsEns, smem);
  cudaGetLastError();
  return b > 0 ? b : 1;
}

void launch_ens_phase_ff(int phase, const FFStep* steps, const int* order, const int* start, int ngroups, int nitems,
                         int blocks, int parity, size_t smem, cudaStream_t st) {
  if (nitems < 1 || blocks < 1) return;
  if (phase == 0) {
    if (smem)
      ens_rhs_ff_kernel<true><<<blocks, dim3(kT, kBY), sizeof(RhsSmem<true>), st>>>(steps, order, start, ngroups, nitems,
                                                                                  parity);
    else
      ens_rhs_ff_kernel<false><<<blocks, dim3(kT, kBY), sizeof(RhsSmem<false>), st>>>(steps, order, start, ngroups,
                                                                                    nitems, parity);
  } else if (phase == 1) {
    ens_x_ff_kernel<<<blocks, kXThreads, smem, st>>>(steps, order, start, ngroups, nitems);
  } else {
    ens_y_ff_kernel<<<blocks, kYThreadsEns, smem, st>>>(steps, order, start, ngroups, nitems, parity);
  }
}

}  // namespace chx
