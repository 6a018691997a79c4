// Batched Crank-Nicolson steps of the two 1D periodic benchmark problems:
//  order 4, hyperdiffusion (Sec. 4.2.1, eq:1d_hyper_scheme), sigma = kappa dt / (2 dx^4):
//    (sigma, -4 sigma, 1 + 6 sigma, -4 sigma, sigma) C^{n+1}
//      = (-sigma, 4 sigma, 1 - 6 sigma, 4 sigma, -sigma) C^n,
//  order 2, diffusion (Sec. 5.3.2, eq5:1ddiffscheme), sigma = kappa dt / (2 dx^2):
//    (-sigma, 1 + 2 sigma, -sigma) C^{n+1} = (sigma, 1 - 2 sigma, sigma) C^n,
// for a batch of systems in the interleaved layout c[i * batch + s].
//
// One thread per system, one forward + backward pass per step (see below for
// the form of the step).  Two ways to hold the matrix, the paper's benchmark
// variants (Sec. 4.3):
//  Constant  factors formed once on the host and shared by every system;
//  Rewrite   every step resets each system's matrix entries in device memory
//            and refactorises them per system (penta_cyclic_refactor /
//            tri_cyclic_refactor), and the sweep reads per-system factors.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "chx_internal.cuh"

using namespace chx;

struct chx_cn1d_plan {
  PlanHdr hdr;
  int order, n, batch, rewrite;
  double sigma;
  double* d_fac;  // Constant: penta 9*(n-2), tri 5*n doubles
  double sinv[4];
  double* d_g;    // forward-sweep scratch, n * batch doubles
  // Rewrite: per-system matrix entries (order + 1 diagonals of n * batch) and a
  // PER_SYSTEM solver plan holding the per-system factors
  double* d_coef;
  chx_penta_plan* penta;
  chx_tri_plan* tri;
};

namespace {

constexpr int kThreads = 128;
constexpr int kU = 8;

// Both schemes have the form A C^{n+1} = B C^n with B = 2I - A (the explicit
// row is twice the identity minus the implicit one), so C^{n+1} = 2 A^{-1} C^n
// - C^n: one solve with right-hand side C^n and a final 2u - C^n, with no
// explicit half to form (penta: 10 FP64 operations per unknown instead of 14,
// tri: 6 instead of 8).  The forward sweep's intermediate goes to the plan's
// scratch g (n * batch doubles, interleaved), the result overwrites c.

// Pentadiagonal (order 4).  Factor rows [ralpha, beta, eps, gam, del, q0, q1,
// G0, G1] over the m = n - 2 rows of the bordered block, then (PER) the 2x2
// tail inverse of each system.
template <bool PER>
__global__ void __launch_bounds__(kThreads) cn_penta_kernel(double* c, double* __restrict__ gs, int n, int batch,
                                                            const double* __restrict__ fac, double s00, double s01,
                                                            double s10, double s11) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const int m = n - 2;
  const size_t B = (size_t)batch;
  const size_t fst = PER ? B : 1, fofs = PER ? (size_t)s : 0;
#define FAC(k, r) __ldg(&fac[((size_t)(k) * m + (r)) * fst + fofs])
  double* pc = c + s;
  double* pg = gs + s;
  double g1 = 0, g2 = 0, t0 = 0, t1 = 0;
  double buf[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) buf[u] = (u < m) ? pc[(size_t)u * B] : 0.0;
  for (int r0 = 0; r0 < m; r0 += kU) {
    double nxt[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + kU + u;
      nxt[u] = (r < m) ? pc[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const double f = buf[u];
        const double g = (f - FAC(2, r) * g2 - FAC(1, r) * g1) * FAC(0, r);
        t0 = fma(FAC(5, r), f, t0);
        t1 = fma(FAC(6, r), f, t1);
        pg[(size_t)r * B] = g;
        g2 = g1;
        g1 = g;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) buf[u] = nxt[u];
  }
  if (PER) {
    const size_t base = (size_t)9 * m * B + (size_t)s;
    s00 = __ldg(&fac[base]);
    s01 = __ldg(&fac[base + B]);
    s10 = __ldg(&fac[base + 2 * B]);
    s11 = __ldg(&fac[base + 3 * B]);
  }
  const double fm = pc[(size_t)m * B], fl = pc[(size_t)(m + 1) * B];
  const double r0v = fm - t0, r1v = fl - t1;
  const double xt0 = s00 * r0v + s01 * r1v, xt1 = s10 * r0v + s11 * r1v;
  pc[(size_t)m * B] = fma(2.0, xt0, -fm);
  pc[(size_t)(m + 1) * B] = fma(2.0, xt1, -fl);
  double x1 = 0, x2 = 0;  // u of rows r+1, r+2
  double gb[kU], cb[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int r = m - 1 - u;
    gb[u] = (r >= 0) ? pg[(size_t)r * B] : 0.0;
    cb[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
  }
  for (int r0 = m - 1; r0 >= 0; r0 -= kU) {
    double gn[kU], cn[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - kU - u;
      gn[u] = (r >= 0) ? pg[(size_t)r * B] : 0.0;
      cn[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        double v = fma(-FAC(7, r), xt0, gb[u]);
        v = fma(-FAC(8, r), xt1, v);
        v = fma(-FAC(4, r), x2, v);
        v = fma(-FAC(3, r), x1, v);
        pc[(size_t)r * B] = fma(2.0, v, -cb[u]);
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      gb[u] = gn[u];
      cb[u] = cn[u];
    }
  }
#undef FAC
}

// Tridiagonal (order 2), Thomas with the Sherman-Morrison correction folded
// into the sweeps as in tri.cu.  Factor rows [rden, a, chat, z, omega].
template <bool PER>
__global__ void __launch_bounds__(kThreads) cn_tri_kernel(double* c, double* __restrict__ gs, int n, int batch,
                                                          const double* __restrict__ fac) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const size_t B = (size_t)batch;
  const size_t fst = PER ? B : 1, fofs = PER ? (size_t)s : 0;
#define FAC(k, r) __ldg(&fac[((size_t)(k) * n + (r)) * fst + fofs])
  double* pc = c + s;
  double* pg = gs + s;
  double d1 = 0, phi = 0;
  double buf[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) buf[u] = (u < n) ? pc[(size_t)u * B] : 0.0;
  for (int r0 = 0; r0 < n; r0 += kU) {
    double nxt[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + kU + u;
      nxt[u] = (r < n) ? pc[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 + u;
      if (r < n) {
        const double dh = fma(-FAC(1, r), d1, buf[u]) * FAC(0, r);
        phi = fma(FAC(4, r), dh, phi);
        pg[(size_t)r * B] = dh;
        d1 = dh;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) buf[u] = nxt[u];
  }
  double y1 = 0;
  double gb[kU], cb[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int r = n - 1 - u;
    gb[u] = (r >= 0) ? pg[(size_t)r * B] : 0.0;
    cb[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
  }
  for (int r0 = n - 1; r0 >= 0; r0 -= kU) {
    double gn[kU], cn[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - kU - u;
      gn[u] = (r >= 0) ? pg[(size_t)r * B] : 0.0;
      cn[u] = (r >= 0) ? pc[(size_t)r * B] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        const double y = fma(-FAC(2, r), y1, gb[u]);
        const double x = fma(-phi, FAC(3, r), y);  // u = A^{-1} C^n
        pc[(size_t)r * B] = fma(2.0, x, -cb[u]);
        y1 = y;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      gb[u] = gn[u];
      cb[u] = cn[u];
    }
  }
#undef FAC
}

// Rewrite mode: every system's matrix entries, diagonal k of row i at
// coef[(k * n + i) * batch + s], set to the scheme's implicit coefficients.
__global__ void cn_reset_matrix_kernel(double* coef, size_t per_diag, int ndiag, double v0, double v1, double v2,
                                       double v3, double v4) {
  const size_t total = per_diag * (size_t)ndiag;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i / per_diag;
    coef[i] = k == 0 ? v0 : k == 1 ? v1 : k == 2 ? v2 : k == 3 ? v3 : v4;
  }
}

void implicit_coefs(int order, double sg, double* v) {
  if (order == 4) {
    v[0] = sg; v[1] = -4.0 * sg; v[2] = 1.0 + 6.0 * sg; v[3] = -4.0 * sg; v[4] = sg;
  } else {
    v[0] = -sg; v[1] = 1.0 + 2.0 * sg; v[2] = -sg; v[3] = 0.0; v[4] = 0.0;
  }
}

}  // namespace

namespace chx {
void penta_plan_free(chx_penta_plan* p);
void tri_plan_free(chx_tri_plan* p);

void* cn1d_inner_plan(chx_cn1d_plan* p) {
  return p->penta ? (void*)p->penta : (void*)p->tri;
}

void cn1d_plan_free(chx_cn1d_plan* p) {
  if (!p) return;
  if (p->d_fac) cudaFree(p->d_fac);
  if (p->d_g) cudaFree(p->d_g);
  if (p->d_coef) cudaFree(p->d_coef);
  if (p->penta) penta_plan_free(p->penta);
  if (p->tri) tri_plan_free(p->tri);
  hdr_free(&p->hdr);
  free(p);
}
}  // namespace chx

static int cn1d_reset_and_factor(chx_cn1d_plan* p, cudaStream_t st) {
  double v[5];
  implicit_coefs(p->order, p->sigma, v);
  const int ndiag = p->order + 1;
  const size_t per = (size_t)p->n * p->batch;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = ceil_div(per * ndiag, (size_t)256);
  const unsigned grid = (unsigned)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
  cn_reset_matrix_kernel<<<grid, 256, 0, st>>>(p->d_coef, per, ndiag, v[0], v[1], v[2], v[3], v[4]);
  int rc = launch_check("cn1d: matrix reset");
  if (rc) return rc;
  const double* D = p->d_coef;
  if (p->order == 4) return penta_cyclic_refactor(p->penta, D, D + per, D + 2 * per, D + 3 * per, D + 4 * per, st);
  return tri_cyclic_refactor(p->tri, D, D + per, D + 2 * per, st);
}

extern "C" int cn1d_plan_create(chx_cn1d_plan** plan, int order, int n, int batch, double l, double kappa, double dt,
                                int rewrite) {
  if (!plan) return fail(CHX_EINVAL, "cn1d_plan_create: null plan pointer");
  *plan = nullptr;
  if (order != 2 && order != 4) return fail(CHX_EINVAL, "cn1d_plan_create: order %d (2 or 4)", order);
  const int nmin = order == 4 ? 6 : 3;
  if (n < nmin || batch < 1 || (rewrite != 0 && rewrite != 1))
    return fail(CHX_EINVAL, "cn1d_plan_create: n %d (>= %d), batch %d (>= 1), rewrite %d (0 or 1)", n, nmin, batch,
                rewrite);
  if (!(l > 0) || !(dt > 0) || !(kappa >= 0) || !isfinite(l) || !isfinite(dt) || !isfinite(kappa))
    return fail(CHX_EINVAL, "cn1d_plan_create: l %g, kappa %g, dt %g", l, kappa, dt);
  chx_cn1d_plan* p = (chx_cn1d_plan*)calloc(1, sizeof(chx_cn1d_plan));
  if (!p) return fail(CHX_ENOMEM, "cn1d_plan_create: plan allocation");
  int rc = hdr_init(&p->hdr, kMagicCn1d);
  if (rc) { cn1d_plan_free(p); return rc; }
  const double dx = l / n;
  p->order = order;
  p->n = n;
  p->batch = batch;
  p->rewrite = rewrite;
  p->sigma = order == 4 ? kappa * dt / (2.0 * dx * dx * dx * dx) : kappa * dt / (2.0 * dx * dx);
  if (cudaMalloc(&p->d_g, (size_t)n * batch * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    p->d_g = nullptr;
    cn1d_plan_free(p);
    return fail(CHX_ENOMEM, "cn1d_plan_create: sweep scratch");
  }
  double v[5];
  implicit_coefs(order, p->sigma, v);
  if (rewrite) {
    const size_t bytes = (size_t)(order + 1) * n * batch * sizeof(double);
    if (cudaMalloc(&p->d_coef, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->d_coef = nullptr;
      cn1d_plan_free(p);
      return fail(CHX_ENOMEM, "cn1d_plan_create: per-system matrix (%zu bytes)", bytes);
    }
    // the solver plan's PER_SYSTEM factorisation needs valid entries: reset them first
    const size_t per = (size_t)n * batch;
    const size_t want = ceil_div(per * (order + 1), (size_t)256);
    cn_reset_matrix_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256>>>(p->d_coef, per, order + 1, v[0], v[1], v[2],
                                                                          v[3], v[4]);
    rc = launch_check("cn1d_plan_create: matrix reset");
    const double* D = p->d_coef;
    if (!rc && order == 4)
      rc = penta_cyclic_factor(&p->penta, n, CHX_COEF_PER_SYSTEM, D, D + per, D + 2 * per, D + 3 * per, D + 4 * per,
                               batch, CHX_F64, nullptr);
    else if (!rc)
      rc = tri_cyclic_factor(&p->tri, n, CHX_COEF_PER_SYSTEM, D, D + per, D + 2 * per, batch, CHX_F64, nullptr);
    if (!rc) rc = chx_sync_status(order == 4 ? (void*)p->penta : (void*)p->tri);
    if (rc) { cn1d_plan_free(p); return rc; }
    *plan = p;
    return CHX_OK;
  }
  std::vector<double> rows(5 * (size_t)n);
  for (int k = 0; k < 5; ++k)
    for (int i = 0; i < n; ++i) rows[(size_t)k * n + i] = v[k];
  double* arr = nullptr;
  size_t cnt = 0;
  if (order == 4) {
    PentaFactors pf;
    rc = penta_factor_host(n, &rows[0], &rows[n], &rows[2 * (size_t)n], &rows[3 * (size_t)n],
                           &rows[4 * (size_t)n], 1, &pf);
    memcpy(p->sinv, pf.sinv, sizeof(p->sinv));
    arr = pf.arr;
    cnt = 9 * (size_t)pf.m;
  } else {
    TriFactors tf;
    rc = tri_factor_host(n, &rows[0], &rows[n], &rows[2 * (size_t)n], 1, &tf);
    arr = tf.arr;
    cnt = 5 * (size_t)n;
  }
  if (rc) { free(arr); cn1d_plan_free(p); return rc; }
  if (cudaMalloc(&p->d_fac, cnt * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    p->d_fac = nullptr;
    free(arr);
    cn1d_plan_free(p);
    return fail(CHX_ENOMEM, "cn1d_plan_create: factor allocation");
  }
  rc = cuda_check(cudaMemcpy(p->d_fac, arr, cnt * sizeof(double), cudaMemcpyHostToDevice), "cn1d_plan_create: upload");
  free(arr);
  if (rc) { cn1d_plan_free(p); return rc; }
  *plan = p;
  return CHX_OK;
}

extern "C" int cn1d_step(chx_cn1d_plan* p, double* c, int nsteps, void* stream) {
  if (!p || p->hdr.magic != kMagicCn1d) return fail(CHX_EINVAL, "cn1d_step: bad plan");
  if (!c || nsteps < 0) return fail(CHX_EINVAL, "cn1d_step: null field or nsteps %d < 0", nsteps);
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blk = balanced_block(p->batch), grid = ceil_div(p->batch, blk);
  for (int k = 0; k < nsteps; ++k) {
    if (p->rewrite) {
      int rc = cn1d_reset_and_factor(p, st);
      if (rc) return rc;
      // the refactor records the inner plan's stream; the sweep follows on `st`
      if (p->order == 4)
        cn_penta_kernel<true><<<grid, blk, 0, st>>>(c, p->d_g, p->n, p->batch, penta_plan_factors(p->penta), 0, 0, 0,
                                                    0);
      else
        cn_tri_kernel<true><<<grid, blk, 0, st>>>(c, p->d_g, p->n, p->batch, tri_plan_factors(p->tri));
    } else if (p->order == 4) {
      cn_penta_kernel<false><<<grid, blk, 0, st>>>(c, p->d_g, p->n, p->batch, p->d_fac, p->sinv[0], p->sinv[1],
                                                   p->sinv[2], p->sinv[3]);
    } else {
      cn_tri_kernel<false><<<grid, blk, 0, st>>>(c, p->d_g, p->n, p->batch, p->d_fac);
    }
  }
  p->hdr.last_stream = st;
  return launch_check("cn1d_step");
}
