// Batched cyclic pentadiagonal solver (Secs. 4.2.2-4.2.5 and 5.4).
//
// One thread per system on the interleaved layout x[i * batch + s], so every
// warp access to row i is one contiguous 256-byte (FP64) segment.  The
// periodic corners are removed by Navon's bordering of the last two unknowns;
// the precomputed bordering vectors are folded into the sweeps so a solve is a
// single forward and a single backward pass over the right-hand side:
//   forward   g_r = (f_r - eps_r g_{r-2} - beta_r g_{r-1}) / alpha_r,
//             t   += q_r f_r                 (t = h^T E^{-1} fhat, q = E^{-T} h)
//   tail      x_tail = S^{-1} (f_tail - t)   (Eq. first_two)
//   backward  x_r = g_r - G_r . x_tail - gam_r x_{r+1} - del_r x_{r+2}
//             (Eq. solve: xhat = E^{-1}(fhat - k x_tail), G = L^{-1} k).
// Factor arrays per row: [ralpha, beta, eps, gam, del, q0, q1, G0, G1].
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "chx_internal.cuh"
#include "mixed.cuh"

using namespace chx;

struct chx_penta_plan {
  PlanHdr hdr;
  int n, m, batch, mode, dtype;
  void* d_fac;        // SHARED/UNIFORM: 9*m values; PER_SYSTEM: (9*m + 4) * batch values (dtype)
  double sinv[4];     // SHARED/UNIFORM tail inverse
  // FP32 sweeps + double-float residual refinement (SHARED/UNIFORM FP64 plans)
  float* d_fac32;     // 9*m floats
  float2* d_coef;     // 5*n double-float pairs: the rows of A for the residual
  float* d_work32;    // n*batch floats
  float sinv32[4];
};

namespace {

constexpr int kThreads = 128;
constexpr int kUnroll = 8;

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Where column (r + o) mod n of row r falls: 0..m-1 -> E/h column, m or m+1 -> tail.
__device__ __forceinline__ int col_of(int r, int o, int n) {
  int c = r + o;
  if (c < 0) c += n;
  if (c >= n) c -= n;
  return c;
}

// ---------------------------------------------------------------------------
// Solve kernel.  TIn: storage of f, TW: storage of the sweep intermediate and of
// x, TC: arithmetic.  For the plain solve all three are the plan dtype and
// in == work (in place).
template <typename TIn, typename TW, typename TC, bool PER>
__global__ void __launch_bounds__(kThreads) penta_solve_kernel(const TIn* in, TW* work, int n, int batch,
                                                               const TC* __restrict__ fac, TC s00, TC s01,
                                                               TC s10, TC s11) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
  const size_t fst = PER ? B : 1, fofs = PER ? (size_t)s : 0;
#define FAC(k, r) ldg(&fac[((size_t)(k) * m + (r)) * fst + fofs])
  const TIn* pin = in + s;
  TW* pw = work + s;
  TC g1 = 0, g2 = 0, t0 = 0, t1 = 0;
  TC buf[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) buf[u] = (u < m) ? (TC)pin[(size_t)u * B] : TC(0);
  for (int r0 = 0; r0 < m; r0 += kUnroll) {
    TC nxt[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 + kUnroll + u;
      nxt[u] = (r < m) ? (TC)pin[(size_t)r * B] : TC(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const TC f = buf[u];
        const TC g = (f - FAC(2, r) * g2 - FAC(1, r) * g1) * FAC(0, r);
        t0 = fma(FAC(5, r), f, t0);
        t1 = fma(FAC(6, r), f, t1);
        pw[(size_t)r * B] = (TW)g;
        g2 = g1;
        g1 = g;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) buf[u] = nxt[u];
  }
  if (PER) {
    const size_t base = (size_t)9 * m * B + (size_t)s;
    s00 = ldg(&fac[base]); s01 = ldg(&fac[base + B]); s10 = ldg(&fac[base + 2 * B]); s11 = ldg(&fac[base + 3 * B]);
  }
  const TC r0v = (TC)pin[(size_t)m * B] - t0, r1v = (TC)pin[(size_t)(m + 1) * B] - t1;
  const TC xt0 = s00 * r0v + s01 * r1v, xt1 = s10 * r0v + s11 * r1v;
  pw[(size_t)m * B] = (TW)xt0;
  pw[(size_t)(m + 1) * B] = (TW)xt1;
  TC x1 = 0, x2 = 0;
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int r = m - 1 - u;
    buf[u] = (r >= 0) ? (TC)pw[(size_t)r * B] : TC(0);
  }
  for (int r0 = m - 1; r0 >= 0; r0 -= kUnroll) {
    TC nxt[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 - kUnroll - u;
      nxt[u] = (r >= 0) ? (TC)pw[(size_t)r * B] : TC(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        TC v = fma(-FAC(7, r), xt0, buf[u]);
        v = fma(-FAC(8, r), xt1, v);
        v = fma(-FAC(3, r), x1, v);
        v = fma(-FAC(4, r), x2, v);
        pw[(size_t)r * B] = (TW)v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) buf[u] = nxt[u];
  }
#undef FAC
}

// ---------------------------------------------------------------------------
// PER_SYSTEM factorisation, one thread per system; coefficients interleaved.
// Forward pass: LU of E (paper factor steps), G = L^{-1} k and y = R^{-T} h in
// registers; backward pass: q = L^{-T} y, S = D - q^T k; tail inverse.
// Only rows 0, 1, m-2 and m-1 of E touch the periodic corners (the k columns,
// the h entries and the wrapped band entries); the rows between take a
// straight-line path with k = h = 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) penta_factor_kernel(const double* __restrict__ a,
                                                                const double* __restrict__ b,
                                                                const double* __restrict__ c,
                                                                const double* __restrict__ d,
                                                                const double* __restrict__ e, int n, int batch,
                                                                T* fac, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
  const double* co[5] = {a + s, b + s, c + s, d + s, e + s};
  T* F = fac + s;
#define FST(k, r) F[((size_t)(k) * m + (r)) * B]
  const double tol = 1e3 * 2.220446049250313e-16;
  double ga1 = 0, ga2 = 0, de1 = 0, de2 = 0;  // gam/del of rows r-1, r-2
  double G01 = 0, G02 = 0, G11 = 0, G12 = 0;  // G rows r-1, r-2
  double y01 = 0, y02 = 0, y11 = 0, y12 = 0;  // y rows r-1, r-2
  bool bad = false;
  // one forward row; b0..b4 the row's entries on E-columns r-2..r+2 (0 off E)
  auto fwd = [&](int r, double b0, double b1, double b2, double b3, double b4, double k0, double k1, double h0,
                 double h1) {
    const double ar = b0;
    const double br = b1 - ar * ga2;
    const double al = b2 - ar * de2 - br * ga1;
    const double scale = fabs(b0) + fabs(b1) + fabs(b2) + fabs(b3) + fabs(b4);
    if (!(fabs(al) > tol * scale)) bad = true;
    const double ra = 1.0 / al;
    const double ga = (b3 - br * de1) * ra;
    const double de = b4 * ra;
    const double G0 = (k0 - ar * G02 - br * G01) * ra;
    const double G1 = (k1 - ar * G12 - br * G11) * ra;
    const double y0 = h0 - ga1 * y01 - de2 * y02;
    const double y1 = h1 - ga1 * y11 - de2 * y12;
    FST(0, r) = (T)ra; FST(1, r) = (T)br; FST(2, r) = (T)ar; FST(3, r) = (T)ga; FST(4, r) = (T)de;
    FST(5, r) = (T)y0; FST(6, r) = (T)y1; FST(7, r) = (T)G0; FST(8, r) = (T)G1;
    ga2 = ga1; ga1 = ga; de2 = de1; de1 = de;
    G02 = G01; G01 = G0; G12 = G11; G11 = G1;
    y02 = y01; y01 = y0; y12 = y11; y11 = y1;
  };
  // a corner row: entries whose column wraps or falls on the tail go to k0/k1
  auto fwd_corner = [&](int r) {
    double bnd[5], k0 = 0, k1 = 0, h0 = 0, h1 = 0;
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      const double v = co[o + 2][(size_t)r * B];
      const int cc = r + o;
      const bool in = cc >= 0 && cc < m;
      bnd[o + 2] = in ? v : 0.0;
      if (!in) {
        if (col_of(r, o, n) == m) k0 += v;
        else k1 += v;
      }
    }
    // h: entries of the last two rows (m, m + 1) on E-column r
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int o = -2; o <= 2; ++o)
        if (col_of(m + q, o, n) == r) (q ? h1 : h0) += co[o + 2][(size_t)(m + q) * B];
    fwd(r, bnd[0], bnd[1], bnd[2], bnd[3], bnd[4], k0, k1, h0, h1);
  };
  const int lo = m < 2 ? m : 2, hi = m - 2 > lo ? m - 2 : lo;  // interior rows [lo, hi)
  for (int r = 0; r < lo; ++r) fwd_corner(r);
  for (int r = lo; r < hi; ++r) {
    const size_t o = (size_t)r * B;
    fwd(r, co[0][o], co[1][o], co[2][o], co[3][o], co[4][o], 0.0, 0.0, 0.0, 0.0);
  }
  for (int r = hi; r < m; ++r) fwd_corner(r);
  double q01 = 0, q02 = 0, q11 = 0, q12 = 0;  // q rows r+1, r+2
  double be1 = 0, ep2 = 0, ep1 = 0;           // beta_{r+1}, eps_{r+2}, eps_{r+1}
  double S00 = 0, S01 = 0, S10 = 0, S11 = 0;  // accumulates q^T k
  auto bwd = [&](int r, bool corner) {
    const double ra = (double)FST(0, r);
    const double q0 = ((double)FST(5, r) - be1 * q01 - ep2 * q02) * ra;
    const double q1 = ((double)FST(6, r) - be1 * q11 - ep2 * q12) * ra;
    FST(5, r) = (T)q0;
    FST(6, r) = (T)q1;
    if (corner) {
      double k0 = 0, k1 = 0;
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        const int cc = r + o;
        if (cc >= 0 && cc < m) continue;
        const double v = co[o + 2][(size_t)r * B];
        if (col_of(r, o, n) == m) k0 += v;
        else k1 += v;
      }
      S00 += q0 * k0; S01 += q0 * k1; S10 += q1 * k0; S11 += q1 * k1;
    }
    q02 = q01; q01 = q0; q12 = q11; q11 = q1;
    ep2 = ep1;
    ep1 = (double)FST(2, r);
    be1 = (double)FST(1, r);
  };
  for (int r = m - 1; r >= hi; --r) bwd(r, true);
  for (int r = hi - 1; r >= lo; --r) bwd(r, false);
  for (int r = lo - 1; r >= 0; --r) bwd(r, true);
  double D00 = 0, D01 = 0, D10 = 0, D11 = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      const int cc = col_of(m + q, o, n);
      const double v = cc >= m ? co[o + 2][(size_t)(m + q) * B] : 0.0;
      if (cc == m) (q ? D10 : D00) += v;
      else if (cc == m + 1) (q ? D11 : D01) += v;
    }
  const double A00 = D00 - S00, A01 = D01 - S01, A10 = D10 - S10, A11 = D11 - S11;
  const double det = A00 * A11 - A01 * A10;
  if (!(fabs(det) > tol * (fabs(A00 * A11) + fabs(A01 * A10)))) bad = true;
  const size_t base = (size_t)9 * m * B;
  F[base] = (T)(A11 / det);
  F[base + B] = (T)(-A01 / det);
  F[base + 2 * B] = (T)(-A10 / det);
  F[base + 3 * B] = (T)(A00 / det);
  if (bad) set_status(status, CHX_ESINGULAR);
#undef FST
}

template <typename T>
int upload_factors(const PentaFactors& pf, void** dst) {
  const size_t cnt = 9 * (size_t)pf.m;
  std::vector<T> h(cnt);
  for (size_t i = 0; i < cnt; ++i) h[i] = (T)pf.arr[i];
  if (cudaMalloc(dst, cnt * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return fail(CHX_ENOMEM, "penta: factor allocation (%zu values)", cnt);
  }
  return cuda_check(cudaMemcpy(*dst, h.data(), cnt * sizeof(T), cudaMemcpyHostToDevice), "penta: factor upload");
}

}  // namespace

namespace chx {
const double* penta_plan_factors(const chx_penta_plan* p) { return (const double*)p->d_fac; }

void penta_plan_free(chx_penta_plan* p) {
  if (!p) return;
  if (p->d_fac) cudaFree(p->d_fac);
  if (p->d_fac32) cudaFree(p->d_fac32);
  if (p->d_coef) cudaFree(p->d_coef);
  if (p->d_work32) cudaFree(p->d_work32);
  hdr_free(&p->hdr);
  free(p);
}
}  // namespace chx

static int launch_per_system_factor(chx_penta_plan* p, const double* a, const double* b, const double* c,
                                    const double* d, const double* e, cudaStream_t st) {
  const unsigned blk = balanced_block(p->batch), grid = ceil_div(p->batch, blk);
  if (p->dtype == CHX_F64)
    penta_factor_kernel<double><<<grid, blk, 0, st>>>(a, b, c, d, e, p->n, p->batch, (double*)p->d_fac,
                                                            p->hdr.d_status);
  else
    penta_factor_kernel<float><<<grid, blk, 0, st>>>(a, b, c, d, e, p->n, p->batch, (float*)p->d_fac,
                                                           p->hdr.d_status);
  p->hdr.last_stream = st;
  return launch_check("penta_factor_kernel");
}

extern "C" int penta_cyclic_factor(chx_penta_plan** plan, int n, int coef_mode, const double* a, const double* b,
                                   const double* c, const double* d, const double* e, int batch, int dtype,
                                   void* stream) {
  if (!plan) return fail(CHX_EINVAL, "penta_cyclic_factor: null plan pointer");
  *plan = nullptr;
  if (n < 5 || batch < 1) return fail(CHX_EINVAL, "penta_cyclic_factor: n = %d (>= 5), batch = %d (>= 1)", n, batch);
  if (dtype != CHX_F64 && dtype != CHX_F32) return fail(CHX_EINVAL, "penta_cyclic_factor: dtype %d", dtype);
  if (coef_mode < CHX_COEF_UNIFORM || coef_mode > CHX_COEF_PER_SYSTEM)
    return fail(CHX_EINVAL, "penta_cyclic_factor: coef_mode %d", coef_mode);
  if (!a || !b || !c || !d || !e) return fail(CHX_EINVAL, "penta_cyclic_factor: null coefficient pointer");
  chx_penta_plan* p = (chx_penta_plan*)calloc(1, sizeof(chx_penta_plan));
  if (!p) return fail(CHX_ENOMEM, "penta_cyclic_factor: plan allocation");
  int rc = hdr_init(&p->hdr, kMagicPenta);
  p->n = n; p->m = n - 2; p->batch = batch; p->mode = coef_mode; p->dtype = dtype;
  if (rc) { penta_plan_free(p); return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  if (coef_mode == CHX_COEF_PER_SYSTEM) {
    const size_t cnt = ((size_t)9 * p->m + 4) * (size_t)batch;
    const size_t esz = dtype == CHX_F64 ? sizeof(double) : sizeof(float);
    if (cudaMalloc(&p->d_fac, cnt * esz) != cudaSuccess) {
      cudaGetLastError();
      p->d_fac = nullptr;
      penta_plan_free(p);
      return fail(CHX_ENOMEM, "penta_cyclic_factor: per-system factors (%zu bytes)", cnt * esz);
    }
    rc = launch_per_system_factor(p, a, b, c, d, e, st);
    if (rc) { penta_plan_free(p); return rc; }
    *plan = p;
    return CHX_OK;
  }
  // UNIFORM / SHARED: host FP64 factorisation.
  std::vector<double> co(5 * (size_t)n);
  const double* src[5] = {a, b, c, d, e};
  for (int k = 0; k < 5; ++k)
    for (int i = 0; i < n; ++i) co[(size_t)k * n + i] = coef_mode == CHX_COEF_UNIFORM ? src[k][0] : src[k][i];
  PentaFactors pf;
  rc = penta_factor_host(n, &co[0], &co[n], &co[2 * (size_t)n], &co[3 * (size_t)n], &co[4 * (size_t)n], 1, &pf);
  if (rc) { penta_plan_free(p); return rc; }
  memcpy(p->sinv, pf.sinv, sizeof(p->sinv));
  for (int i = 0; i < 4; ++i) p->sinv32[i] = (float)pf.sinv[i];
  rc = dtype == CHX_F64 ? upload_factors<double>(pf, &p->d_fac) : upload_factors<float>(pf, &p->d_fac);
  if (!rc && dtype == CHX_F64) {
    void* f32 = nullptr;
    rc = upload_factors<float>(pf, &f32);
    p->d_fac32 = (float*)f32;
    if (!rc) {
      std::vector<float2> cff(co.size());
      for (size_t k = 0; k < co.size(); ++k) cff[k] = split_ff(co[k]);
      if (cudaMalloc(&p->d_coef, cff.size() * sizeof(float2)) != cudaSuccess ||
          cudaMalloc(&p->d_work32, (size_t)n * batch * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(CHX_ENOMEM, "penta_cyclic_factor: refinement storage");
      } else {
        rc = cuda_check(cudaMemcpy(p->d_coef, cff.data(), cff.size() * sizeof(float2), cudaMemcpyHostToDevice),
                        "penta: coefficient upload");
      }
    }
  }
  free(pf.arr);
  if (rc) { penta_plan_free(p); return rc; }
  p->hdr.last_stream = st;
  *plan = p;
  return CHX_OK;
}

extern "C" int penta_cyclic_refactor(chx_penta_plan* p, const double* a, const double* b, const double* c,
                                     const double* d, const double* e, void* stream) {
  if (!p || p->hdr.magic != kMagicPenta) return fail(CHX_EINVAL, "penta_cyclic_refactor: bad plan");
  if (p->mode != CHX_COEF_PER_SYSTEM) return fail(CHX_EINVAL, "penta_cyclic_refactor: PER_SYSTEM plans only");
  if (!a || !b || !c || !d || !e) return fail(CHX_EINVAL, "penta_cyclic_refactor: null coefficient pointer");
  return launch_per_system_factor(p, a, b, c, d, e, (cudaStream_t)stream);
}

extern "C" int penta_cyclic_solve_batched(chx_penta_plan* p, void* rhs, int batch, int refine, void* stream) {
  if (!p || p->hdr.magic != kMagicPenta) return fail(CHX_EINVAL, "penta_cyclic_solve_batched: bad plan");
  if (!rhs) return fail(CHX_EINVAL, "penta_cyclic_solve_batched: null rhs");
  if (batch < 1 || batch > p->batch)
    return fail(CHX_EINVAL, "penta_cyclic_solve_batched: batch %d outside [1, %d]", batch, p->batch);
  if (p->mode == CHX_COEF_PER_SYSTEM && batch != p->batch)
    return fail(CHX_EINVAL, "penta_cyclic_solve_batched: PER_SYSTEM batch must equal the factor batch %d", p->batch);
  if (refine && p->dtype != CHX_F64) return fail(CHX_EINVAL, "penta_cyclic_solve_batched: refine needs an FP64 plan");
  if (refine && p->mode == CHX_COEF_PER_SYSTEM)
    return fail(CHX_EUNSUPPORTED, "penta_cyclic_solve_batched: refine with PER_SYSTEM coefficients");
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blk = balanced_block(batch), grid = ceil_div(batch, blk);
  const double* S = p->sinv;
  const float* S32 = p->sinv32;
  if (refine) {
    launch_penta_refine_ff((double*)rhs, p->d_work32, p->n, batch, p->d_fac32, p->d_coef, S32, st);
  } else if (p->dtype == CHX_F64) {
    double* x = (double*)rhs;
    if (p->mode == CHX_COEF_PER_SYSTEM)
      penta_solve_kernel<double, double, double, true><<<grid, blk, 0, st>>>(x, x, p->n, batch,
                                                                                 (const double*)p->d_fac, 0, 0, 0, 0);
    else
      penta_solve_kernel<double, double, double, false><<<grid, blk, 0, st>>>(
          x, x, p->n, batch, (const double*)p->d_fac, S[0], S[1], S[2], S[3]);
  } else {
    float* x = (float*)rhs;
    if (p->mode == CHX_COEF_PER_SYSTEM)
      penta_solve_kernel<float, float, float, true><<<grid, blk, 0, st>>>(x, x, p->n, batch,
                                                                              (const float*)p->d_fac, 0, 0, 0, 0);
    else
      penta_solve_kernel<float, float, float, false><<<grid, blk, 0, st>>>(
          x, x, p->n, batch, (const float*)p->d_fac, S32[0], S32[1], S32[2], S32[3]);
  }
  p->hdr.last_stream = st;
  return launch_check("penta_cyclic_solve_batched");
}
