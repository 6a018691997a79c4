// Status handling, plan bookkeeping and the host FP64 factorisations shared by
// the solver and Cahn-Hilliard plans.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chx_internal.cuh"

namespace chx {

static thread_local char g_last_error[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CHX_OK;
  return fail(CHX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int launch_check(const char* what) { return cuda_check(cudaGetLastError(), what); }

unsigned balanced_block(size_t threads) {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& n = sms[dev & 63];
  if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    n = 152;
  }
  return threads < (size_t)128 * 16 * n ? 32u : 128u;
}

int hdr_init(PlanHdr* h, uint32_t magic) {
  h->magic = magic;
  h->d_status = nullptr;
  h->last_stream = nullptr;
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->d_status = nullptr;
    return fail(CHX_ENOMEM, "plan status word allocation failed");
  }
  return cuda_check(cudaMemset(h->d_status, 0, sizeof(int)), "status word init");
}

void hdr_free(PlanHdr* h) {
  if (h->d_status) cudaFree(h->d_status);
  h->d_status = nullptr;
  h->magic = 0;
}

static const double kEps = 2.220446049250313e-16;
static const double kPivotTol = 1e3 * kEps;

// -------------------------------------------------------------------------
// Cyclic pentadiagonal: Navon bordering + LU without pivoting (Secs. 4.2.2-3).
int penta_factor_host(int n, const double* a, const double* b, const double* c, const double* d,
                      const double* e, size_t cs, PentaFactors* out) {
  if (n < 5) return fail(CHX_EINVAL, "penta: n = %d < 5", n);
  const int m = n - 2;
  const double* co[5] = {a, b, c, d, e};
  std::vector<double> band(5 * (size_t)m, 0.0), k0(m, 0.0), k1(m, 0.0);
  // Rows 0..m-1: entries on the first m columns form the band of E; the two
  // tail columns (n-2, n-1) form k (Eq. xhat).
  for (int r = 0; r < m; ++r) {
    for (int o = -2; o <= 2; ++o) {
      double v = co[o + 2][(size_t)r * cs];
      int col = r + o;
      if (col >= 0 && col < m) {
        band[(size_t)(o + 2) * m + r] = v;
      } else {
        if (col < 0) col += n;
        if (col == m) k0[r] += v;
        else k1[r] += v;
      }
    }
  }
  double* arr = (double*)calloc(9 * (size_t)m, sizeof(double));
  if (!arr) return fail(CHX_ENOMEM, "penta: host factor allocation");
  double *ra = arr, *be = arr + m, *ep = arr + 2 * m, *ga = arr + 3 * m, *de = arr + 4 * m;
  double *q0 = arr + 5 * m, *q1 = arr + 6 * m, *G0 = arr + 7 * m, *G1 = arr + 8 * m;
  const double *Ea = band.data(), *Eb = Ea + m, *Ec = Eb + m, *Ed = Ec + m, *Ee = Ed + m;
  std::vector<double> alpha(m);
  for (int r = 0; r < m; ++r) {
    double ar = Ea[r];
    double br = Eb[r] - (r >= 2 ? ar * ga[r - 2] : 0.0);
    double al = Ec[r] - (r >= 2 ? ar * de[r - 2] : 0.0) - (r >= 1 ? br * ga[r - 1] : 0.0);
    double scale = fabs(Ea[r]) + fabs(Eb[r]) + fabs(Ec[r]) + fabs(Ed[r]) + fabs(Ee[r]);
    if (!(fabs(al) > kPivotTol * scale)) {
      free(arr);
      return fail(CHX_ESINGULAR, "penta: pivot %d of %d is %.3e (row scale %.3e)", r, m, al, scale);
    }
    alpha[r] = al;
    ra[r] = 1.0 / al;
    be[r] = br;
    ep[r] = ar;
    ga[r] = (Ed[r] - (r >= 1 ? br * de[r - 1] : 0.0)) / al;
    de[r] = Ee[r] / al;
  }
  // G = L^{-1} k (forward substitution with L = (alpha, beta, eps)).
  for (int r = 0; r < m; ++r) {
    double g0 = k0[r], g1 = k1[r];
    if (r >= 2) { g0 -= ep[r] * G0[r - 2]; g1 -= ep[r] * G1[r - 2]; }
    if (r >= 1) { g0 -= be[r] * G0[r - 1]; g1 -= be[r] * G1[r - 1]; }
    G0[r] = g0 * ra[r];
    G1[r] = g1 * ra[r];
  }
  // Last two rows: their E-columns form h^T, their tail columns D.
  std::vector<double> h0(m, 0.0), h1(m, 0.0);
  double D[2][2] = {{0, 0}, {0, 0}};
  for (int q = 0; q < 2; ++q) {
    int r = m + q;
    for (int o = -2; o <= 2; ++o) {
      double v = co[o + 2][(size_t)r * cs];
      int col = r + o;
      if (col >= n) col -= n;
      if (col < m) (q ? h1 : h0)[col] += v;
      else D[q][col - m] += v;
    }
  }
  // q = E^{-T} h: R^T y = h (forward), then L^T q = y (backward).
  for (int r = 0; r < m; ++r) {
    double y0 = h0[r], y1 = h1[r];
    if (r >= 1) { y0 -= ga[r - 1] * q0[r - 1]; y1 -= ga[r - 1] * q1[r - 1]; }
    if (r >= 2) { y0 -= de[r - 2] * q0[r - 2]; y1 -= de[r - 2] * q1[r - 2]; }
    q0[r] = y0;
    q1[r] = y1;
  }
  for (int r = m - 1; r >= 0; --r) {
    double y0 = q0[r], y1 = q1[r];
    if (r + 1 < m) { y0 -= be[r + 1] * q0[r + 1]; y1 -= be[r + 1] * q1[r + 1]; }
    if (r + 2 < m) { y0 -= ep[r + 2] * q0[r + 2]; y1 -= ep[r + 2] * q1[r + 2]; }
    q0[r] = y0 * ra[r];
    q1[r] = y1 * ra[r];
  }
  // S = D - q^T k (k is sparse but a dense dot keeps this plain).
  double S[2][2];
  for (int q = 0; q < 2; ++q) {
    const double* qq = q ? q1 : q0;
    double s0 = 0.0, s1 = 0.0;
    for (int r = 0; r < m; ++r) { s0 += qq[r] * k0[r]; s1 += qq[r] * k1[r]; }
    S[q][0] = D[q][0] - s0;
    S[q][1] = D[q][1] - s1;
  }
  double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
  double dsc = fabs(S[0][0] * S[1][1]) + fabs(S[0][1] * S[1][0]);
  if (!(fabs(det) > kPivotTol * dsc)) {
    free(arr);
    return fail(CHX_ESINGULAR, "penta: bordering 2x2 determinant %.3e (scale %.3e)", det, dsc);
  }
  out->n = n;
  out->m = m;
  out->arr = arr;
  out->sinv[0] = S[1][1] / det;
  out->sinv[1] = -S[0][1] / det;
  out->sinv[2] = -S[1][0] / det;
  out->sinv[3] = S[0][0] / det;
  return CHX_OK;
}

// -------------------------------------------------------------------------
// Cyclic tridiagonal: Thomas with pre-factorisation + Sherman-Morrison (Sec. 5.3).
int tri_factor_host(int n, const double* a, const double* b, const double* c, size_t cs, TriFactors* out) {
  if (n < 3) return fail(CHX_EINVAL, "tri: n = %d < 3", n);
  const double a0 = a[0], b0 = b[0], cN = c[(size_t)(n - 1) * cs];
  if (!(fabs(b0) > 0.0)) return fail(CHX_ESINGULAR, "tri: b_1 = 0");
  double* arr = (double*)calloc(5 * (size_t)n, sizeof(double));
  if (!arr) return fail(CHX_ENOMEM, "tri: host factor allocation");
  double *rd = arr, *aa = arr + n, *ch = arr + 2 * n, *z = arr + 3 * n, *om = arr + 4 * n;
  for (int i = 0; i < n; ++i) {
    double ai = i > 0 ? a[(size_t)i * cs] : 0.0;  // a_1 moved into u v^T
    double ci = i < n - 1 ? c[(size_t)i * cs] : 0.0;  // c_N moved into u v^T
    double bi = b[(size_t)i * cs];
    if (i == 0) bi = 2.0 * b0;
    if (i == n - 1) bi = bi + a0 * cN / b0;
    double den = bi - (i > 0 ? ai * ch[i - 1] : 0.0);
    double scale = fabs(ai) + fabs(bi) + fabs(ci);
    if (!(fabs(den) > kPivotTol * scale)) {
      free(arr);
      return fail(CHX_ESINGULAR, "tri: pivot %d is %.3e (row scale %.3e)", i, den, scale);
    }
    rd[i] = 1.0 / den;
    aa[i] = ai;
    ch[i] = ci / den;
  }
  // z = A'^{-1} u, u = (-b_1, 0, .., 0, c_N).
  for (int i = 0; i < n; ++i) {
    double ui = (i == 0 ? -b0 : 0.0) + (i == n - 1 ? cN : 0.0);
    z[i] = (ui - (i > 0 ? aa[i] * z[i - 1] : 0.0)) * rd[i];
  }
  for (int i = n - 2; i >= 0; --i) z[i] -= ch[i] * z[i + 1];
  double r = a0 / b0;
  double vz = z[0] - r * z[n - 1];
  double den = 1.0 + vz;
  if (!(fabs(den) > kPivotTol * (1.0 + fabs(vz)))) {
    free(arr);
    return fail(CHX_ESINGULAR, "tri: Sherman-Morrison denominator 1 + v.z = %.3e", den);
  }
  // y_1 = sum_k w_k dhat_k with w = R^{-T} e_1 (R: unit upper bidiagonal chat).
  double w = 1.0;
  for (int k = 0; k < n; ++k) {
    om[k] = w / den;
    w = -ch[k] * w;
  }
  om[n - 1] -= r / den;
  out->n = n;
  out->arr = arr;
  return CHX_OK;
}

// -------------------------------------------------------------------------
int band_factor_host(int m, double a, double b, double c, double d, double e, double* ra, double* be,
                     double* ga, double* de) {
  for (int r = 0; r < m; ++r) {
    double ar = r >= 2 ? a : 0.0, br0 = r >= 1 ? b : 0.0;
    double dr = r + 1 < m ? d : 0.0, er = r + 2 < m ? e : 0.0;
    double br = br0 - (r >= 2 ? ar * ga[r - 2] : 0.0);
    double al = c - (r >= 2 ? ar * de[r - 2] : 0.0) - (r >= 1 ? br * ga[r - 1] : 0.0);
    double scale = fabs(ar) + fabs(br0) + fabs(c) + fabs(dr) + fabs(er);
    if (!(fabs(al) > kPivotTol * scale)) return fail(CHX_ESINGULAR, "band: pivot %d is %.3e", r, al);
    ra[r] = 1.0 / al;
    be[r] = br;
    ga[r] = (dr - (r >= 1 ? br * de[r - 1] : 0.0)) / al;
    de[r] = er / al;
  }
  return CHX_OK;
}

void band_solve_host(int m, double a, const double* ra, const double* be, const double* ga, const double* de,
                     const double* f, double* x) {
  for (int r = 0; r < m; ++r) {
    double s = f[r];
    if (r >= 2) s -= a * x[r - 2];
    if (r >= 1) s -= be[r] * x[r - 1];
    x[r] = s * ra[r];
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = x[r];
    if (r + 1 < m) s -= ga[r] * x[r + 1];
    if (r + 2 < m) s -= de[r] * x[r + 2];
    x[r] = s;
  }
}

int dense_inverse_host(int k, const double* A, double* Ainv) {
  std::vector<double> M((size_t)k * 2 * k, 0.0);
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < k; ++j) M[(size_t)i * 2 * k + j] = A[(size_t)i * k + j];
    M[(size_t)i * 2 * k + k + i] = 1.0;
  }
  double amax = 0.0;
  for (int i = 0; i < k * k; ++i) amax = fmax(amax, fabs(A[i]));
  for (int col = 0; col < k; ++col) {
    int piv = col;
    for (int r = col + 1; r < k; ++r)
      if (fabs(M[(size_t)r * 2 * k + col]) > fabs(M[(size_t)piv * 2 * k + col])) piv = r;
    double p = M[(size_t)piv * 2 * k + col];
    if (!(fabs(p) > kPivotTol * amax)) return fail(CHX_ESINGULAR, "dense inverse: pivot %.3e", p);
    if (piv != col)
      for (int j = 0; j < 2 * k; ++j) {
        double t = M[(size_t)piv * 2 * k + j];
        M[(size_t)piv * 2 * k + j] = M[(size_t)col * 2 * k + j];
        M[(size_t)col * 2 * k + j] = t;
      }
    double ip = 1.0 / p;
    for (int j = 0; j < 2 * k; ++j) M[(size_t)col * 2 * k + j] *= ip;
    for (int r = 0; r < k; ++r) {
      if (r == col) continue;
      double f = M[(size_t)r * 2 * k + col];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * k; ++j) M[(size_t)r * 2 * k + j] -= f * M[(size_t)col * 2 * k + j];
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Ainv[(size_t)i * k + j] = M[(size_t)i * 2 * k + k + j];
  return CHX_OK;
}

// Per-type destructors live with their plans.
void penta_plan_free(chx_penta_plan* p);
void tri_plan_free(chx_tri_plan* p);
void ch_plan_free(chx_ch_plan* p);
void ens_free(chx_ens* e);
void ch1d_plan_free(chx_ch1d_plan* p);
void cn1d_plan_free(chx_cn1d_plan* p);
void* cn1d_inner_plan(chx_cn1d_plan* p);

}  // namespace chx

using namespace chx;

extern "C" const char* chx_status_string(int s) {
  switch (s) {
    case CHX_OK: return "CHX_OK";
    case CHX_EINVAL: return "CHX_EINVAL";
    case CHX_ESINGULAR: return "CHX_ESINGULAR";
    case CHX_ENONFINITE: return "CHX_ENONFINITE";
    case CHX_ENOMEM: return "CHX_ENOMEM";
    case CHX_ECUDA: return "CHX_ECUDA";
    case CHX_ETIMEOUT: return "CHX_ETIMEOUT";
    case CHX_EUNSUPPORTED: return "CHX_EUNSUPPORTED";
    default: return "CHX_UNKNOWN";
  }
}

extern "C" const char* chx_last_error(void) { return g_last_error; }

extern "C" int chx_version(void) { return 10000; }

extern "C" int chx_coarsening_rate(const double* t, const double* F, int count, double* beta) {
  if (!t || !F || !beta || count < 3) return fail(CHX_EINVAL, "chx_coarsening_rate: null pointer or count %d < 3", count);
  for (int k = 1; k < count; ++k)
    if (!(t[k] > t[k - 1])) return fail(CHX_EINVAL, "chx_coarsening_rate: times not increasing at %d", k);
  for (int k = 0; k < count; ++k)
    if (!(F[k] != 0.0) || !isfinite(F[k])) return fail(CHX_EINVAL, "chx_coarsening_rate: F[%d] = %g", k, F[k]);
  // derivative of the quadratic through three neighbouring samples: centred
  // inside, one-sided at the two ends (second order on uneven spacing)
  for (int k = 0; k < count; ++k) {
    const int c = k == 0 ? 1 : (k == count - 1 ? count - 2 : k);
    const double h1 = t[c] - t[c - 1], h2 = t[c + 1] - t[c];
    const double f0 = F[c - 1], f1 = F[c], f2 = F[c + 1];
    double d;
    if (k == 0)
      d = -(2 * h1 + h2) / (h1 * (h1 + h2)) * f0 + (h1 + h2) / (h1 * h2) * f1 - h1 / (h2 * (h1 + h2)) * f2;
    else if (k == count - 1)
      d = h2 / (h1 * (h1 + h2)) * f0 - (h1 + h2) / (h1 * h2) * f1 + (2 * h2 + h1) / (h2 * (h1 + h2)) * f2;
    else
      d = (h1 * h1 * f2 - h2 * h2 * f0 + (h2 * h2 - h1 * h1) * f1) / (h1 * h2 * (h1 + h2));
    beta[k] = -(t[k] / F[k]) * d;
  }
  return CHX_OK;
}

extern "C" int chx_sync_status(void* plan) {
  if (!plan) return fail(CHX_EINVAL, "chx_sync_status: null plan");
  PlanHdr* h = (PlanHdr*)plan;
  if (h->magic != kMagicPenta && h->magic != kMagicTri && h->magic != kMagicCh && h->magic != kMagicEns &&
      h->magic != kMagicCh1d && h->magic != kMagicCn1d)
    return fail(CHX_EINVAL, "chx_sync_status: not a chx plan");
  if (h->magic == kMagicCn1d) {  // a Rewrite plan's per-system factorisation flags its own solver plan
    void* inner = cn1d_inner_plan((chx_cn1d_plan*)plan);
    if (inner) {
      int rc = chx_sync_status(inner);
      if (rc) return rc;
    }
  }
  int rc = cuda_check(cudaStreamSynchronize(h->last_stream), "chx_sync_status: stream synchronize");
  if (rc) return rc;
  int st = 0;
  rc = cuda_check(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "chx_sync_status: read");
  if (rc) return rc;
  if (st != 0) {
    cudaMemset(h->d_status, 0, sizeof(int));
    return fail(st, "device reported %s", chx_status_string(st));
  }
  return CHX_OK;
}

extern "C" void chx_plan_destroy(void* plan) {
  if (!plan) return;
  PlanHdr* h = (PlanHdr*)plan;
  switch (h->magic) {
    case kMagicPenta: penta_plan_free((chx_penta_plan*)plan); break;
    case kMagicTri: tri_plan_free((chx_tri_plan*)plan); break;
    case kMagicCh: ch_plan_free((chx_ch_plan*)plan); break;
    case kMagicEns: ens_free((chx_ens*)plan); break;
    case kMagicCh1d: ch1d_plan_free((chx_ch1d_plan*)plan); break;
    case kMagicCn1d: cn1d_plan_free((chx_cn1d_plan*)plan); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput: sixteen independent chains per thread and a loop body
// of 64 FMAs, so the FP64 pipe rather than the FMA latency or the loop's own
// instructions sets the rate; the result feeds a sink only if it takes an
// impossible value, which keeps the chains live.  The same chains do not always
// issue at the same rate: on one GB300 at 2070 MHz they ran at 627 G per second
// (2.0 per clock per SM) with the trip count passed at run time, and at 528 G
// (1.68 per clock, the rate of plain FP64 adds and multiplies there) with it
// fixed at compile time.  So the rate is taken over two operand forms with a
// run-time trip count, and the larger one is reported.
namespace {
constexpr int kRateChains = 16, kRateUnroll = 4, kRateThreads = 256, kRateBlocksPerSM = 8;
// FROM_MEMORY: the multiplier and addend are loaded into registers; else
// they are kernel parameters
template <bool FROM_MEMORY>
__global__ void fp64_fma_rate_kernel(double* sink, const double* __restrict__ cst, double mul, double add,
                                     int iters) {
  const double m = FROM_MEMORY ? cst[0] : mul;
  const double a = FROM_MEMORY ? cst[1] : add;
  double v[kRateChains];
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) v[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kRateUnroll; ++j)
#pragma unroll
      for (int k = 0; k < kRateChains; ++k) v[k] = fma(v[k], m, a);
  }
  double t = 0;
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) t += v[k];
  if (t == -1.0) *sink = t;
}
}  // namespace

extern "C" int chx_fp64_fma_rate(double* gops_out, void* stream) {
  if (!gops_out) return fail(CHX_EINVAL, "chx_fp64_fma_rate: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "chx_fp64_fma_rate: device");
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "chx_fp64_fma_rate: SMs");
  if (rc) return rc;
  double* buf = nullptr;  // [0] the sink, [1], [2] the multiplier and addend
  cudaEvent_t a = nullptr, b = nullptr;
  const double consts[2] = {0.999999999, 1e-12};
  if ((rc = cuda_check(cudaMalloc(&buf, 3 * sizeof(double)), "chx_fp64_fma_rate: scratch")) ||
      (rc = cuda_check(cudaMemcpy(buf + 1, consts, sizeof(consts), cudaMemcpyHostToDevice), "chx_fp64_fma_rate: constants")) ||
      (rc = cuda_check(cudaEventCreate(&a), "chx_fp64_fma_rate: event")) ||
      (rc = cuda_check(cudaEventCreate(&b), "chx_fp64_fma_rate: event"))) {
    cudaFree(buf);
    if (a) cudaEventDestroy(a);
    return rc;
  }
  const unsigned blocks = (unsigned)sms * kRateBlocksPerSM;
  const int iters = 1024, timed = 2;
  double best = 0.0;
  for (int form = 0; form < 2 && !rc; ++form) {
    auto launch = [&] {
      if (form) fp64_fma_rate_kernel<true><<<blocks, kRateThreads, 0, st>>>(buf, buf + 1, consts[0], consts[1], iters);
      else fp64_fma_rate_kernel<false><<<blocks, kRateThreads, 0, st>>>(buf, buf + 1, consts[0], consts[1], iters);
    };
    launch();  // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < timed; ++r) launch();
    cudaEventRecord(b, st);
    rc = cuda_check(cudaEventSynchronize(b), "chx_fp64_fma_rate: run");
    float ms = 0.f;
    if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, a, b), "chx_fp64_fma_rate: timing");
    const double fmas = (double)timed * blocks * kRateThreads * kRateChains * kRateUnroll * iters;
    if (!rc && ms > 0.f) best = std::max(best, fmas / (ms * 1e-3) / 1e9);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (rc) return rc;
  *gops_out = best;
  return CHX_OK;
}

