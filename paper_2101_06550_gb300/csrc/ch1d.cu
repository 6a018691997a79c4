// Batched 1D Cahn-Hilliard (Sec. 6.2.1, eq6:1Dnumerical):
//   (I + sigma delta^4) C^{n+1} = C^n + alpha delta^2 (C^3 - C)^n,
//   sigma = gamma dt / dx^4, alpha = dt / dx^2, periodic,
// for a batch of independent simulations in the interleaved layout
// c[i * batch + s] (the thesis runs 2^20 of them at N = 256, Sec. 6.2.3).
//
// One thread per simulation.  The right-hand side is formed inside the forward
// sweep of the cyclic pentadiagonal solve (Navon bordering folded in, as in
// penta.cu) from a three-point register window of C, so a step is a single
// in-place forward + backward pass: the forward sweep overwrites row r with its
// intermediate once f_r is formed, the window keeps the values the next rows
// still need, and C_0 is kept for the last row's periodic neighbour.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "chx_internal.cuh"

using namespace chx;

struct chx_ch1d_plan {
  PlanHdr hdr;
  int n, batch;
  double alpha;
  double* d_fac;  // 9*(n-2): ralpha, beta, eps, gam, del, q0, q1, G0, G1
  double sinv[4];
};

namespace {

constexpr int kThreads = 128;
constexpr int kU = 8;

__device__ __forceinline__ double nlin(double c) { return c * fma(c, c, -1.0); }

__global__ void __launch_bounds__(kThreads) ch1d_step_kernel(double* c, int n, int batch, double alpha,
                                                             const double* __restrict__ fac, double s00, double s01,
                                                             double s10, double s11) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
#define FAC(k, r) __ldg(&fac[(size_t)(k) * m + (r)])
  double* pc = c + s;
  const double c0 = pc[0];
  const double Nlast = nlin(pc[(size_t)(n - 1) * B]);
  double Nprev = Nlast, ccur = c0, Ncur = nlin(c0);
  double g1 = 0, g2 = 0, t0 = 0, t1 = 0;
  // rows r + 1 (the window's leading edge), prefetched kU ahead; r + 1 <= m < n
  double buf[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) buf[u] = (u + 1 <= m) ? pc[(size_t)(u + 1) * B] : 0.0;
  for (int r0 = 0; r0 < m; r0 += kU) {
    double nxt[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + kU + u;
      nxt[u] = (r + 1 <= m) ? pc[(size_t)(r + 1) * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const double cn1 = buf[u];
        const double Nn1 = nlin(cn1);
        const double f = fma(alpha, fma(-2.0, Ncur, Nprev) + Nn1, ccur);
        const double g = (f - FAC(2, r) * g2 - FAC(1, r) * g1) * FAC(0, r);
        t0 = fma(FAC(5, r), f, t0);
        t1 = fma(FAC(6, r), f, t1);
        pc[(size_t)r * B] = g;  // row r of C is no longer read from memory
        g2 = g1;
        g1 = g;
        Nprev = Ncur;
        Ncur = Nn1;
        ccur = cn1;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) buf[u] = nxt[u];
  }
  // tail rows m = n-2 (ccur, Ncur) and m+1 = n-1
  const double cl = pc[(size_t)(m + 1) * B];
  const double fm = fma(alpha, fma(-2.0, Ncur, Nprev) + Nlast, ccur);
  const double fl = fma(alpha, fma(-2.0, Nlast, Ncur) + nlin(c0), cl);
  const double r0v = fm - t0, r1v = fl - t1;
  const double xt0 = s00 * r0v + s01 * r1v, xt1 = s10 * r0v + s11 * r1v;
  pc[(size_t)m * B] = xt0;
  pc[(size_t)(m + 1) * B] = xt1;
  double x1 = 0, x2 = 0;
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int r = m - 1 - u;
    buf[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
  }
  for (int r0 = m - 1; r0 >= 0; r0 -= kU) {
    double nxt[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - kU - u;
      nxt[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        double v = fma(-FAC(7, r), xt0, buf[u]);
        v = fma(-FAC(8, r), xt1, v);
        v = fma(-FAC(3, r), x1, v);
        v = fma(-FAC(4, r), x2, v);
        pc[(size_t)r * B] = v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) buf[u] = nxt[u];
  }
#undef FAC
}

}  // namespace

namespace chx {
void ch1d_plan_free(chx_ch1d_plan* p) {
  if (!p) return;
  if (p->d_fac) cudaFree(p->d_fac);
  hdr_free(&p->hdr);
  free(p);
}
}  // namespace chx

extern "C" int ch1d_plan_create(chx_ch1d_plan** plan, int n, int batch, double l, double gamma, double dt) {
  if (!plan) return fail(CHX_EINVAL, "ch1d_plan_create: null plan pointer");
  *plan = nullptr;
  if (n < 8 || batch < 1) return fail(CHX_EINVAL, "ch1d_plan_create: n %d (>= 8), batch %d (>= 1)", n, batch);
  if (!(l > 0) || !(dt > 0) || !(gamma >= 0) || !isfinite(l) || !isfinite(dt) || !isfinite(gamma))
    return fail(CHX_EINVAL, "ch1d_plan_create: l %g, gamma %g, dt %g", l, gamma, dt);
  chx_ch1d_plan* p = (chx_ch1d_plan*)calloc(1, sizeof(chx_ch1d_plan));
  if (!p) return fail(CHX_ENOMEM, "ch1d_plan_create: plan allocation");
  int rc = hdr_init(&p->hdr, kMagicCh1d);
  if (rc) { ch1d_plan_free(p); return rc; }
  const double dx = l / n;
  const double sigma = gamma * dt / (dx * dx * dx * dx);
  p->n = n;
  p->batch = batch;
  p->alpha = dt / (dx * dx);
  const double co[5] = {sigma, -4.0 * sigma, 1.0 + 6.0 * sigma, -4.0 * sigma, sigma};
  std::vector<double> rows(5 * (size_t)n);
  for (int k = 0; k < 5; ++k)
    for (int i = 0; i < n; ++i) rows[(size_t)k * n + i] = co[k];
  PentaFactors pf;
  rc = penta_factor_host(n, &rows[0], &rows[n], &rows[2 * (size_t)n], &rows[3 * (size_t)n], &rows[4 * (size_t)n], 1,
                         &pf);
  if (rc) { ch1d_plan_free(p); return rc; }
  memcpy(p->sinv, pf.sinv, sizeof(p->sinv));
  const size_t bytes = 9 * (size_t)pf.m * sizeof(double);
  if (cudaMalloc(&p->d_fac, bytes) != cudaSuccess) {
    cudaGetLastError();
    p->d_fac = nullptr;
    free(pf.arr);
    ch1d_plan_free(p);
    return fail(CHX_ENOMEM, "ch1d_plan_create: factor allocation");
  }
  rc = cuda_check(cudaMemcpy(p->d_fac, pf.arr, bytes, cudaMemcpyHostToDevice), "ch1d_plan_create: upload");
  free(pf.arr);
  if (rc) { ch1d_plan_free(p); return rc; }
  *plan = p;
  return CHX_OK;
}

extern "C" int ch1d_step(chx_ch1d_plan* p, double* c, int nsteps, void* stream) {
  if (!p || p->hdr.magic != kMagicCh1d) return fail(CHX_EINVAL, "ch1d_step: bad plan");
  if (!c || nsteps < 0) return fail(CHX_EINVAL, "ch1d_step: null field or nsteps %d < 0", nsteps);
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blk = balanced_block(p->batch), grid = ceil_div(p->batch, blk);
  for (int k = 0; k < nsteps; ++k)
    ch1d_step_kernel<<<grid, blk, 0, st>>>(c, p->n, p->batch, p->alpha, p->d_fac, p->sinv[0], p->sinv[1],
                                                p->sinv[2], p->sinv[3]);
  p->hdr.last_stream = st;
  return launch_check("ch1d_step");
}
