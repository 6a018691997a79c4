// Batched cyclic tridiagonal solver (Sec. 5.3: cuThomasConstantBatch with the
// Sherman-Morrison treatment of the periodic corners).
//
// One thread per system, interleaved layout x[i * batch + s].  z = A'^{-1} u is
// formed once at factor time (the paper's "second solve, performed once").  The
// scalar (v.y)/(1 + v.z) needs y_1, which a plain Thomas back sweep produces
// last; it is instead accumulated in the forward sweep as a dot product of dhat
// with precomputed weights omega (y_1 = w^T dhat, w = R^{-T} e_1), so the
// correction x = y - phi z is applied inside the single back sweep:
//   forward   dhat_i = (f_i - a_i dhat_{i-1}) * rden_i,   phi += omega_i dhat_i
//   backward  y_i = dhat_i - chat_i y_{i+1},              x_i = y_i - phi z_i.
// Factor arrays per row: [rden, a, chat, z, omega].
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "chx_internal.cuh"

using namespace chx;

struct chx_tri_plan {
  PlanHdr hdr;
  int n, batch, mode, dtype;
  void* d_fac;  // SHARED/UNIFORM: 5*n values; PER_SYSTEM: 5*n*batch values (dtype)
};

namespace {

constexpr int kThreads = 128;
constexpr int kUnroll = 8;

template <typename T, bool PER>
__global__ void __launch_bounds__(kThreads) tri_solve_kernel(T* x, int n, int batch, const T* __restrict__ fac) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const size_t B = (size_t)batch;
  const size_t fst = PER ? B : 1, fofs = PER ? (size_t)s : 0;
#define FAC(k, r) __ldg(&fac[((size_t)(k) * n + (r)) * fst + fofs])
  T* p = x + s;
  T d1 = 0, phi = 0;
  T buf[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) buf[u] = (u < n) ? p[(size_t)u * B] : T(0);
  for (int r0 = 0; r0 < n; r0 += kUnroll) {
    T nxt[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 + kUnroll + u;
      nxt[u] = (r < n) ? p[(size_t)r * B] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 + u;
      if (r < n) {
        const T dh = fma(-FAC(1, r), d1, buf[u]) * FAC(0, r);
        phi = fma(FAC(4, r), dh, phi);
        p[(size_t)r * B] = dh;
        d1 = dh;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) buf[u] = nxt[u];
  }
  T y1 = 0;
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int r = n - 1 - u;
    buf[u] = (r >= 0) ? p[(size_t)r * B] : T(0);
  }
  for (int r0 = n - 1; r0 >= 0; r0 -= kUnroll) {
    T nxt[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 - kUnroll - u;
      nxt[u] = (r >= 0) ? p[(size_t)r * B] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        const T y = fma(-FAC(2, r), y1, buf[u]);
        p[(size_t)r * B] = fma(-phi, FAC(3, r), y);
        y1 = y;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) buf[u] = nxt[u];
  }
#undef FAC
}

// PER_SYSTEM factorisation: Thomas factors of A', z = A'^{-1} u, weights omega.
template <typename T>
__global__ void __launch_bounds__(kThreads) tri_factor_kernel(const double* __restrict__ a,
                                                              const double* __restrict__ b,
                                                              const double* __restrict__ c, int n, int batch,
                                                              T* fac, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= batch) return;
  const size_t B = (size_t)batch;
  T* F = fac + s;
#define FST(k, r) F[((size_t)(k) * n + (r)) * B]
  const double tol = 1e3 * 2.220446049250313e-16;
  const double a0 = a[s], b0 = b[s], cN = c[(size_t)(n - 1) * B + s];
  bool bad = !(fabs(b0) > 0.0);
  const double rb = bad ? 0.0 : a0 / b0;
  double ch1 = 0, z1 = 0;
  for (int i = 0; i < n; ++i) {
    const double ai = i > 0 ? a[(size_t)i * B + s] : 0.0;
    const double ci = i < n - 1 ? c[(size_t)i * B + s] : 0.0;
    double bi = b[(size_t)i * B + s];
    if (i == 0) bi = 2.0 * b0;
    if (i == n - 1) bi = bi + a0 * cN / b0;
    const double den = bi - ai * ch1;
    if (!(fabs(den) > tol * (fabs(ai) + fabs(bi) + fabs(ci)))) bad = true;
    const double rd = 1.0 / den;
    const double ch = ci * rd;
    const double ui = (i == 0 ? -b0 : 0.0) + (i == n - 1 ? cN : 0.0);
    const double zh = (ui - ai * z1) * rd;
    FST(0, i) = (T)rd; FST(1, i) = (T)ai; FST(2, i) = (T)ch; FST(3, i) = (T)zh;
    ch1 = ch;
    z1 = zh;
  }
  double zn = 0, zlast = 0, zfirst = 0;
  for (int i = n - 1; i >= 0; --i) {
    const double z = (double)FST(3, i) - (double)FST(2, i) * zn;
    FST(3, i) = (T)z;
    if (i == n - 1) zlast = z;
    zfirst = z;
    zn = z;
  }
  const double vz = zfirst - rb * zlast;
  const double den = 1.0 + vz;
  if (!(fabs(den) > tol * (1.0 + fabs(vz)))) bad = true;
  const double rden = 1.0 / den;  // one division, not one per row
  double w = 1.0;
  for (int k = 0; k < n; ++k) {
    double om = w * rden;
    if (k == n - 1) om -= rb * rden;
    FST(4, k) = (T)om;
    w = -(double)FST(2, k) * w;
  }
  if (bad) set_status(status, CHX_ESINGULAR);
#undef FST
}

}  // namespace

namespace chx {
const double* tri_plan_factors(const chx_tri_plan* p) { return (const double*)p->d_fac; }

void tri_plan_free(chx_tri_plan* p) {
  if (!p) return;
  if (p->d_fac) cudaFree(p->d_fac);
  hdr_free(&p->hdr);
  free(p);
}
}  // namespace chx

static int launch_tri_factor(chx_tri_plan* p, const double* a, const double* b, const double* c,
                             cudaStream_t st) {
  const unsigned blk = balanced_block(p->batch), grid = ceil_div(p->batch, blk);
  if (p->dtype == CHX_F64)
    tri_factor_kernel<double><<<grid, blk, 0, st>>>(a, b, c, p->n, p->batch, (double*)p->d_fac,
                                                          p->hdr.d_status);
  else
    tri_factor_kernel<float><<<grid, blk, 0, st>>>(a, b, c, p->n, p->batch, (float*)p->d_fac,
                                                         p->hdr.d_status);
  p->hdr.last_stream = st;
  return launch_check("tri_factor_kernel");
}

extern "C" int tri_cyclic_factor(chx_tri_plan** plan, int n, int coef_mode, const double* a, const double* b,
                                 const double* c, int batch, int dtype, void* stream) {
  if (!plan) return fail(CHX_EINVAL, "tri_cyclic_factor: null plan pointer");
  *plan = nullptr;
  if (n < 3 || batch < 1) return fail(CHX_EINVAL, "tri_cyclic_factor: n = %d (>= 3), batch = %d (>= 1)", n, batch);
  if (dtype != CHX_F64 && dtype != CHX_F32) return fail(CHX_EINVAL, "tri_cyclic_factor: dtype %d", dtype);
  if (coef_mode < CHX_COEF_UNIFORM || coef_mode > CHX_COEF_PER_SYSTEM)
    return fail(CHX_EINVAL, "tri_cyclic_factor: coef_mode %d", coef_mode);
  if (!a || !b || !c) return fail(CHX_EINVAL, "tri_cyclic_factor: null coefficient pointer");
  chx_tri_plan* p = (chx_tri_plan*)calloc(1, sizeof(chx_tri_plan));
  if (!p) return fail(CHX_ENOMEM, "tri_cyclic_factor: plan allocation");
  int rc = hdr_init(&p->hdr, kMagicTri);
  p->n = n; p->batch = batch; p->mode = coef_mode; p->dtype = dtype;
  if (rc) { tri_plan_free(p); return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t esz = dtype == CHX_F64 ? sizeof(double) : sizeof(float);
  if (coef_mode == CHX_COEF_PER_SYSTEM) {
    const size_t cnt = (size_t)5 * n * batch;
    if (cudaMalloc(&p->d_fac, cnt * esz) != cudaSuccess) {
      cudaGetLastError();
      p->d_fac = nullptr;
      tri_plan_free(p);
      return fail(CHX_ENOMEM, "tri_cyclic_factor: per-system factors (%zu bytes)", cnt * esz);
    }
    rc = launch_tri_factor(p, a, b, c, st);
    if (rc) { tri_plan_free(p); return rc; }
    *plan = p;
    return CHX_OK;
  }
  std::vector<double> co(3 * (size_t)n);
  const double* src[3] = {a, b, c};
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < n; ++i) co[(size_t)k * n + i] = coef_mode == CHX_COEF_UNIFORM ? src[k][0] : src[k][i];
  TriFactors tf;
  rc = tri_factor_host(n, &co[0], &co[n], &co[2 * (size_t)n], 1, &tf);
  if (rc) { tri_plan_free(p); return rc; }
  const size_t cnt = 5 * (size_t)n;
  if (cudaMalloc(&p->d_fac, cnt * esz) != cudaSuccess) {
    cudaGetLastError();
    p->d_fac = nullptr;
    free(tf.arr);
    tri_plan_free(p);
    return fail(CHX_ENOMEM, "tri_cyclic_factor: factor allocation");
  }
  if (dtype == CHX_F64) {
    rc = cuda_check(cudaMemcpy(p->d_fac, tf.arr, cnt * esz, cudaMemcpyHostToDevice), "tri: factor upload");
  } else {
    std::vector<float> h(cnt);
    for (size_t i = 0; i < cnt; ++i) h[i] = (float)tf.arr[i];
    rc = cuda_check(cudaMemcpy(p->d_fac, h.data(), cnt * esz, cudaMemcpyHostToDevice), "tri: factor upload");
  }
  free(tf.arr);
  if (rc) { tri_plan_free(p); return rc; }
  p->hdr.last_stream = st;
  *plan = p;
  return CHX_OK;
}

extern "C" int tri_cyclic_refactor(chx_tri_plan* p, const double* a, const double* b, const double* c,
                                   void* stream) {
  if (!p || p->hdr.magic != kMagicTri) return fail(CHX_EINVAL, "tri_cyclic_refactor: bad plan");
  if (p->mode != CHX_COEF_PER_SYSTEM) return fail(CHX_EINVAL, "tri_cyclic_refactor: PER_SYSTEM plans only");
  if (!a || !b || !c) return fail(CHX_EINVAL, "tri_cyclic_refactor: null coefficient pointer");
  return launch_tri_factor(p, a, b, c, (cudaStream_t)stream);
}

extern "C" int tri_cyclic_solve_batched(chx_tri_plan* p, void* rhs, int batch, void* stream) {
  if (!p || p->hdr.magic != kMagicTri) return fail(CHX_EINVAL, "tri_cyclic_solve_batched: bad plan");
  if (!rhs) return fail(CHX_EINVAL, "tri_cyclic_solve_batched: null rhs");
  if (batch < 1 || batch > p->batch)
    return fail(CHX_EINVAL, "tri_cyclic_solve_batched: batch %d outside [1, %d]", batch, p->batch);
  if (p->mode == CHX_COEF_PER_SYSTEM && batch != p->batch)
    return fail(CHX_EINVAL, "tri_cyclic_solve_batched: PER_SYSTEM batch must equal the factor batch %d", p->batch);
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blk = balanced_block(batch), grid = ceil_div(batch, blk);
  if (p->dtype == CHX_F64) {
    if (p->mode == CHX_COEF_PER_SYSTEM)
      tri_solve_kernel<double, true><<<grid, blk, 0, st>>>((double*)rhs, p->n, batch, (const double*)p->d_fac);
    else
      tri_solve_kernel<double, false><<<grid, blk, 0, st>>>((double*)rhs, p->n, batch, (const double*)p->d_fac);
  } else {
    if (p->mode == CHX_COEF_PER_SYSTEM)
      tri_solve_kernel<float, true><<<grid, blk, 0, st>>>((float*)rhs, p->n, batch, (const float*)p->d_fac);
    else
      tri_solve_kernel<float, false><<<grid, blk, 0, st>>>((float*)rhs, p->n, batch, (const float*)p->d_fac);
  }
  p->hdr.last_stream = st;
  return launch_check("tri_cyclic_solve_batched");
}
