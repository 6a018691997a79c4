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
#include "chgroup.cuh"
#include "ff.cuh"

namespace chx {
namespace {

constexpr int kT = 32, kBY = 8, kSolveThreads = 128;

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

// L'(u) = (E + W) + rho (N + S) + kap C on shared-memory ff tiles; for a
// square cell (rho = 1, kap = -4) the scalings are exact and skipped.
template <int LD, bool kIso>
__device__ __forceinline__ ff lap_ff(const ff (*t)[LD], int y, int x, ff rho, ff kap) {
  ff a = ff_add(t[y][x - 1], t[y][x + 1]);
  const ff b = ff_add(t[y - 1][x], t[y + 1][x]);
  if (kIso) return ff_add(ff_add(a, b), ff_scale2(t[y][x], -4.f));
  a = ff_add(a, ff_mul(rho, b));
  return ff_add(a, ff_mul(kap, t[y][x]));
}

// Right-hand side of Eq. 3.1 in double-float: r = k2 L'(M) - k1 (C^n - C^{n-1}),
// M = C^3 - C - gl L'(Cbar), in one pass over 32 x 32 tiles (M formed on the
// tile and a 1-point halo ring): whole 32-column rows per warp while staging,
// j along the warp for the output, whose transposed stores are then coalesced
// without a staging tile.  (The FP64 step splits this into two passes to save
// the ring's FP64 work; here the ring costs issue slots on the FP32 pipes.)
//
// NOISE (Cahn-Hilliard-Cook, Sec. 7.7): the forcing term (2/3) dt eta is
// formed in FP64 on the otherwise idle FP64 unit (one subtraction and one FMA
// per direction) from caller-given or pre-drawn deviates, and added as a
// double-float pair.
template <bool kIso, bool NOISE = false>
__global__ void __launch_bounds__(kT* kBY) ch_rhs_ff_kernel(const double* __restrict__ cn,
                                                            const double* __restrict__ cp, float* __restrict__ rhi,
                                                            float* __restrict__ rlo, int nx, int ny, int G, float2 rho2,
                                                            float2 kap2, const float2* __restrict__ glff, float2 k12,
                                                            float2 k22, const double* __restrict__ dev = nullptr,
                                                            double nkx = 0, double nky = 0) {
  __shared__ ff s_cn[kT + 4][kT + 5];
  __shared__ ff s_cb[kT + 4][kT + 5];
  __shared__ ff s_m[kT + 2][kT + 3];
  __shared__ ff s_nz[NOISE ? kT : 1][kT + 1];
  const int z = blockIdx.z;
  const ff rho = ffc(rho2), kap = ffc(kap2), gl = ffc(glff[z]), k1 = ffc(k12), k2 = ffc(k22);
  cn += (size_t)z * nx * ny;
  cp += (size_t)z * nx * ny;
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int tid = threadIdx.y * kT + threadIdx.x;
  auto stage = [&](int ly, int lx) {
    const int gi = wrap_near(i0 - 2 + lx, nx), gj = wrap_near(j0 - 2 + ly, ny);
    const size_t p = (size_t)gj * nx + gi;
    const ff a = d2ff(cn[p]), b = d2ff(cp[p]);
    s_cn[ly][lx] = a;
    s_cb[ly][lx] = ff_sub(ff_scale2(a, 2.f), b);
  };
  for (int ly = threadIdx.y; ly < kT + 4; ly += kBY) stage(ly, threadIdx.x);
  if (tid < 4 * (kT + 4)) stage(tid >> 2, kT + (tid & 3));
  if (NOISE) {
    const size_t N = (size_t)nx * ny;
    const double* rx = dev + (size_t)z * 2 * N;
    const double* ry = rx + N;
    for (int lj = threadIdx.y; lj < kT; lj += kBY) {
      const int li = threadIdx.x, gi = i0 + li, gj = j0 + lj;
      double v = 0;
      if (gi < nx && gj < ny) {
        const size_t q = (size_t)gj * nx + gi;
        const size_t qw = (size_t)gj * nx + (gi == 0 ? nx - 1 : gi - 1);
        const size_t qs = (size_t)(gj == 0 ? ny - 1 : gj - 1) * nx + gi;
        v = fma(nkx, rx[q] - rx[qw], nky * (ry[q] - ry[qs]));
      }
      s_nz[lj][li] = d2ff(v);
    }
  }
  __syncthreads();
  auto mstage = [&](int ly, int lx) {
    const ff l = lap_ff<kT + 5, kIso>(s_cb, ly, lx, rho, kap);
    const ff c = s_cn[ly][lx];
    const ff nl = ff_mul(c, ff_add_f(ff_mul(c, c), -1.f));
    s_m[ly - 1][lx - 1] = ff_sub(nl, ff_mul(gl, l));
  };
  for (int ly = 1 + threadIdx.y; ly <= kT + 2; ly += kBY) mstage(ly, 1 + threadIdx.x);
  if (tid < 2 * (kT + 2)) mstage(1 + (tid >> 1), kT + 1 + (tid & 1));
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int li = threadIdx.y + k * kBY, lj = threadIdx.x;  // output (i0 + li, j0 + lj)
    const int ly = lj + 1, lx = li + 1;
    const ff l = lap_ff<kT + 3, kIso>(s_m, ly, lx, rho, kap);
    const ff diff = ff_sub(s_cb[ly + 1][lx + 1], s_cn[ly + 1][lx + 1]);  // C^n - C^{n-1}
    ff v = ff_sub(ff_mul(k2, l), ff_mul(k1, diff));
    if (NOISE) v = ff_add(v, s_nz[lj][li]);
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) {
      const size_t q = (size_t)gi * G * ny + (size_t)z * ny + gj;
      rhi[q] = v.hi;
      rlo[q] = v.lo;
    }
  }
}

__device__ __forceinline__ float corr32(const float* __restrict__ vw, const float* __restrict__ tau, int m, int P,
                                        int nsys, int s, int r, int j) {
  const int sn = s + 1 == P ? 0 : s + 1, sp = s == 0 ? P - 1 : s - 1;
  const size_t S = (size_t)nsys;
  float c = __ldg(&vw[r]) * tau[(size_t)(4 * sn + 0) * S + j];
  c = fmaf(__ldg(&vw[m + r]), tau[(size_t)(4 * sn + 1) * S + j], c);
  c = fmaf(__ldg(&vw[2 * m + r]), tau[(size_t)(4 * sp + 2) * S + j], c);
  c = fmaf(__ldg(&vw[3 * m + r]), tau[(size_t)(4 * sp + 3) * S + j], c);
  return c;
}

// A x0 for the ADI row (a, -4a, 1 + 6a, -4a, a): x0 + a * delta^4 x0, the fourth
// difference formed with error-free sums.
__device__ __forceinline__ ff adi_apply_ff(float w0, float w1, float w2, float w3, float w4, ff a) {
  const ff s2 = two_sum(w0, w4);
  const ff s1 = two_sum(w1, w3);
  ff d = ff_sub(s2, ff_scale2(s1, 4.f));
  d = ff_add(d, two_prod(6.f, w2));
  return ff_add_f(ff_mul(a, d), w2);
}

// Refinement residual on tiles of 32 rows x 32 systems: the first FP32
// solution x0 = y1 - spike correction is formed once per element of the tile
// and its 2-row halo and staged in shared memory; then rho = f - A x0 in
// double-float for the tile's points.  Writes rho's high part (the right-hand
// side of the FP32 correction solve) and x0.  Element (row i, system j) at
// [i*ld + j] (+ blockIdx.z * fz); grid (systems / 32, n / 32, Z), block 32 x 8.
__global__ void __launch_bounds__(kT* kBY) ch_resid_ff_kernel(
    const float* __restrict__ fhi, const float* __restrict__ flo, const float* __restrict__ y1,
    const float* __restrict__ t1, float* __restrict__ x0out, float* __restrict__ rho, int ld, int nsys, int n,
    DirView<float> D, const float2* __restrict__ aff, size_t fz, size_t ybz) {
  __shared__ float sx[kT + 4][kT + 1];
  const int m = D.m, P = D.P;
  const int j = blockIdx.x * kT + threadIdx.x;
  const int i0 = blockIdx.y * kT;
  const size_t off = blockIdx.z * fz;
  fhi += off;
  flo += off;
  y1 += off;
  x0out += off;
  rho += off;
  t1 += blockIdx.z * ybz;
  const bool live = j < nsys;
  const int slot = blockIdx.z + (live ? j : 0) / D.spp;
  const float* vw = D.vw + (size_t)slot * 4 * m;
  const size_t S = (size_t)nsys;
  // a warp's rows share threadIdx.y, so the segment (and its four reduced
  // unknowns) changes warp-uniformly and rarely: load them once per segment
  int cs = -1;
  float ta = 0.f, tb = 0.f, tc = 0.f, td = 0.f;
  for (int ly = threadIdx.y; ly < kT + 4; ly += kBY) {
    float v = 0.f;
    if (live) {
      int i = i0 - 2 + ly;
      i = i < 0 ? i + n : (i >= n ? i - n : i);
      int s, r;
      seg_row(i, m, D.rm, s, r);
      if (s != cs) {
        cs = s;
        const int sn = s + 1 == P ? 0 : s + 1, sp = s == 0 ? P - 1 : s - 1;
        ta = t1[(size_t)(4 * sn) * S + j];
        tb = t1[(size_t)(4 * sn + 1) * S + j];
        tc = t1[(size_t)(4 * sp + 2) * S + j];
        td = t1[(size_t)(4 * sp + 3) * S + j];
      }
      float c = __ldg(&vw[r]) * ta;
      c = fmaf(__ldg(&vw[m + r]), tb, c);
      c = fmaf(__ldg(&vw[2 * m + r]), tc, c);
      c = fmaf(__ldg(&vw[3 * m + r]), td, c);
      v = y1[(size_t)i * ld + j] - c;
    }
    sx[ly][threadIdx.x] = v;
  }
  __syncthreads();
  if (!live) return;
  const ff a = ffc(aff[slot]);
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int ly = threadIdx.y + k * kBY, i = i0 + ly;
    if (i >= n) break;
    const float* col = &sx[ly][threadIdx.x];
    const ff ax = adi_apply_ff(col[0], col[kT + 1], col[2 * (kT + 1)], col[3 * (kT + 1)], col[4 * (kT + 1)], a);
    const size_t p = (size_t)i * ld + j;
    rho[p] = ff_sub(ff{fhi[p], flo[p]}, ax).hi;
    x0out[p] = col[2 * (kT + 1)];
  }
}

// x sweep result w = x0 + delta as an exact double-float pair, transposed back
// to row-major (w[j*nx + i]).
__global__ void __launch_bounds__(kT* kBY) ch_xfinish_ff_kernel(const float* __restrict__ y1,
                                                                const float* __restrict__ t1,
                                                                const float* __restrict__ y2,
                                                                const float* __restrict__ t2, DirView<float> D,
                                                                float* __restrict__ whi, float* __restrict__ wlo,
                                                                int nx, int ny, int G) {
  __shared__ ff s_t[kT][kT + 1];
  const int z = blockIdx.z, m = D.m, P = D.P;
  const float* vw = D.vw + (size_t)z * 4 * m;
  const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kT;
  const int j = j0 + threadIdx.x;
  const size_t ld = (size_t)G * ny;
  const int sys = z * ny + j;
  const size_t S = (size_t)G * ny;
  int cs = -1;  // the correction's reduced unknowns, loaded once per segment (warp-uniform)
  float ta = 0.f, tb = 0.f, tc = 0.f, td = 0.f;
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int li = threadIdx.y + k * kBY, i = i0 + li;
    if (i < nx && j < ny) {
      int s, r;
      seg_row(i, m, D.rm, s, r);
      if (s != cs) {
        cs = s;
        const int sn = s + 1 == P ? 0 : s + 1, sp = s == 0 ? P - 1 : s - 1;
        ta = t2[(size_t)(4 * sn) * S + sys];
        tb = t2[(size_t)(4 * sn + 1) * S + sys];
        tc = t2[(size_t)(4 * sp + 2) * S + sys];
        td = t2[(size_t)(4 * sp + 3) * S + sys];
      }
      float c = __ldg(&vw[r]) * ta;
      c = fmaf(__ldg(&vw[m + r]), tb, c);
      c = fmaf(__ldg(&vw[2 * m + r]), tc, c);
      c = fmaf(__ldg(&vw[3 * m + r]), td, c);
      const float x0 = y1[(size_t)i * ld + sys];  // corrected first solution
      const float dl = y2[(size_t)i * ld + sys] - c;
      s_t[li][threadIdx.x] = two_sum(x0, dl);
    }
  }
  __syncthreads();
  whi += (size_t)z * nx * ny;
  wlo += (size_t)z * nx * ny;
#pragma unroll
  for (int k = 0; k < kT / kBY; ++k) {
    const int lj = threadIdx.y + k * kBY, li = threadIdx.x;
    const int gi = i0 + li, gj = j0 + lj;
    if (gi < nx && gj < ny) {
      const ff v = s_t[li][lj];
      whi[(size_t)gj * nx + gi] = v.hi;
      wlo[(size_t)gj * nx + gi] = v.lo;
    }
  }
}

// C^{n+1} = 2 C^n - C^{n-1} + v with v = x0 + delta (exact pair, added in FP64).
__global__ void __launch_bounds__(kSolveThreads) ch_update_ff_kernel(const float* __restrict__ y1,
                                                                     const float* __restrict__ t1,
                                                                     const float* __restrict__ y2,
                                                                     const float* __restrict__ t2, DirView<float> D,
                                                                     double* cn, double* cp, int nx, int ny,
                                                                     int keep_roles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, z = blockIdx.z, m = D.m, P = D.P;
  const float* vw = D.vw + (size_t)z * 4 * m;
  if (i >= nx) return;
  const int s = j / m, r = j - s * m;
  const size_t p = (size_t)z * nx * ny + (size_t)j * nx + i;
  t1 += (size_t)z * 4 * P * nx;
  t2 += (size_t)z * 4 * P * nx;
  const float x0 = y1[p];  // corrected first solution
  const float dl = y2[p] - corr32(vw, t2, m, P, nx, s, r, i);
  const ff v = two_sum(x0, dl);
  const double a = cn[p], b = cp[p];
  const double nxt = fma(2.0, a, -b) + ff2d(v);
  if (keep_roles) {
    cp[p] = a;
    cn[p] = nxt;
  } else {
    cp[p] = nxt;
  }
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

}  // namespace

void launch_ch_rhs_ff(const double* cn, const double* cp, float* rhi, float* rlo, int nx, int ny, int G,
                      const FFConst& k, const float2* glff, const double* noise, double nkx, double nky,
                      cudaStream_t st) {
  const dim3 grid(ceil_div(nx, kT), ceil_div(ny, kT), G), block(kT, kBY);
  const bool iso = k.rho.x == 1.f && k.rho.y == 0.f;
  if (noise && iso)
    ch_rhs_ff_kernel<true, true><<<grid, block, 0, st>>>(cn, cp, rhi, rlo, nx, ny, G, k.rho, k.kap, glff, k.k1, k.k2,
                                                         noise, nkx, nky);
  else if (noise)
    ch_rhs_ff_kernel<false, true><<<grid, block, 0, st>>>(cn, cp, rhi, rlo, nx, ny, G, k.rho, k.kap, glff, k.k1, k.k2,
                                                          noise, nkx, nky);
  else if (iso)
    ch_rhs_ff_kernel<true><<<grid, block, 0, st>>>(cn, cp, rhi, rlo, nx, ny, G, k.rho, k.kap, glff, k.k1, k.k2);
  else
    ch_rhs_ff_kernel<false><<<grid, block, 0, st>>>(cn, cp, rhi, rlo, nx, ny, G, k.rho, k.kap, glff, k.k1, k.k2);
}

void launch_resid_ff(const float* fhi, const float* flo, const float* y1, const float* t1, float* x0, float* rho,
                     int ld, int nsys, int n, const DirView<float>& D, const float2* aff, int Z, size_t fz, size_t ybz,
                     cudaStream_t st) {
  ch_resid_ff_kernel<<<dim3(ceil_div(nsys, kT), ceil_div(n, kT), Z), dim3(kT, kBY), 0, st>>>(fhi, flo, y1, t1, x0, rho,
                                                                                           ld, nsys, n, D, aff, fz, ybz);
}

void launch_ch_xfinish_ff(const float* y1, const float* t1, const float* y2, const float* t2, const DirView<float>& D,
                          float* whi, float* wlo, int nx, int ny, int G, cudaStream_t st) {
  const dim3 grid(ceil_div(nx, kT), ceil_div(ny, kT), G), block(kT, kBY);
  ch_xfinish_ff_kernel<<<grid, block, 0, st>>>(y1, t1, y2, t2, D, whi, wlo, nx, ny, G);
}

void launch_ch_update_ff(const float* y1, const float* t1, const float* y2, const float* t2, const DirView<float>& D,
                         double* cn, double* cp, int nx, int ny, int G, int keep_roles, cudaStream_t st) {
  ch_update_ff_kernel<<<dim3(ceil_div(nx, kSolveThreads), ny, G), kSolveThreads, 0, st>>>(y1, t1, y2, t2, D, cn, cp,
                                                                                         nx, ny, keep_roles);
}

void launch_penta_refine_ff(double* x, float* work, int n, int batch, const float* fac32, const float2* coef_ff,
                            const float* s32, cudaStream_t st) {
  const unsigned blk = balanced_block(batch), grid = ceil_div(batch, blk);
  penta_solve_f32_from_f64_kernel<<<grid, blk, 0, st>>>(x, work, n, batch, fac32, s32[0], s32[1], s32[2],
                                                                   s32[3]);
  penta_refine_ff_kernel<<<grid, blk, 0, st>>>(x, work, n, batch, fac32, coef_ff, s32[0], s32[1], s32[2],
                                                         s32[3]);
}

}  // namespace chx
