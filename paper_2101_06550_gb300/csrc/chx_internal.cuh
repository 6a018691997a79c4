// Internal declarations shared by the chx translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/chx.h"

namespace chx {

// Every plan starts with this header so chx_sync_status / chx_plan_destroy can
// take any plan type.
enum : uint32_t { kMagicPenta = 0x70656e74u, kMagicTri = 0x74726964u, kMagicCh = 0x63686164u, kMagicEns = 0x656e7362u,
                  kMagicCh1d = 0x63683164u, kMagicCn1d = 0x636e3164u };

struct PlanHdr {
  uint32_t magic;
  int* d_status;              // first device-side error, CHX_OK when clean
  cudaStream_t last_stream;   // stream of the most recent enqueue
};

// Records a detail message for chx_last_error() and returns `status`.
int fail(int status, const char* fmt, ...);
// Checks a CUDA runtime result; on failure records it and returns CHX_ECUDA.
int cuda_check(cudaError_t e, const char* what);
// cuda_check(cudaGetLastError()) after a launch.
int launch_check(const char* what);

int hdr_init(PlanHdr* h, uint32_t magic);
void hdr_free(PlanHdr* h);

// Device-side error recording: the first non-zero code wins.
__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Threads per block for one-thread-per-system kernels, whose time is set by the
// busiest SM.  With few blocks per SM, 128-thread blocks leave some SMs a whole
// block ahead of the rest (65536 threads = 512 blocks on 152 SMs: 4 on some,
// 3 on others, 84% balance); single-warp blocks spread the warps to within one
// of each other (96%).  Many blocks balance by themselves and keep 128.
unsigned balanced_block(size_t threads);

// ---------------------------------------------------------------------------
// Host FP64 factorisation of one cyclic pentadiagonal system (Secs. 4.2.2-4.2.3).
// Output arrays (each m = n-2 long): ralpha = 1/alpha, beta, eps (= a on rows
// r >= 2), gam, del (LU of the leading block E), q0, q1 (q = E^{-T} h), G0, G1
// (G = L^{-1} k), and sinv = inverse of the 2x2 tail matrix D - h^T E^{-1} k.
// coef(i, o) gives the coefficient of row i at offset o in [-2, 2].
struct PentaFactors {
  int n = 0, m = 0;
  double* arr = nullptr;  // 9 * m doubles: ralpha, beta, eps, gam, del, q0, q1, G0, G1
  double sinv[4] = {0, 0, 0, 0};
};
int penta_factor_host(int n, const double* a, const double* b, const double* c, const double* d,
                      const double* e, size_t cs, PentaFactors* out);

// Host FP64 factorisation of one cyclic tridiagonal system (Sec. 5.3): per-row
// arrays rden = 1/(b'_i - a_i chat_{i-1}), a, chat, z = A'^{-1} u and
// omega (weights giving phi = (v.y)/(1 + v.z) as a dot product with dhat).
struct TriFactors {
  int n = 0;
  double* arr = nullptr;  // 5 * n doubles: rden, a, chat, z, omega
};
int tri_factor_host(int n, const double* a, const double* b, const double* c, size_t cs, TriFactors* out);

// Device factor storage of an FP64 plan (PER_SYSTEM: interleaved per system,
// followed for the pentadiagonal plan by the 4 tail-inverse entries per system).
const double* penta_plan_factors(const chx_penta_plan* p);
const double* tri_plan_factors(const chx_tri_plan* p);

// Cahn-Hilliard-Cook deviates for G consecutive simulations sim0.. (noise.cu);
// the step index comes from *d_step when d_step is not null.
int launch_noise_normals(double* rho, int nx, int ny, int G, uint64_t seed, uint64_t sim0, uint64_t step,
                         const uint64_t* d_step, cudaStream_t st);
// *d_step += 1, and *d_step = v, on the stream.
int launch_step_advance(uint64_t* d_step, cudaStream_t st);
int launch_step_set(uint64_t* d_step, uint64_t v, cudaStream_t st);

// Plain non-cyclic pentadiagonal LU (paper factor steps) of the m x m Toeplitz
// band (a, b, c, d, e); ralpha, beta, gam, del of length m.
int band_factor_host(int m, double a, double b, double c, double d, double e, double* ralpha, double* beta,
                     double* gam, double* del);
// Solve with the factors above (host, FP64).
void band_solve_host(int m, double a, const double* ralpha, const double* beta, const double* gam,
                     const double* del, const double* f, double* x);
// Dense inverse by Gaussian elimination with partial pivoting (host, FP64).
int dense_inverse_host(int k, const double* A, double* Ainv);

}  // namespace chx
