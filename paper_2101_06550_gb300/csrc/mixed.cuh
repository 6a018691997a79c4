// Launchers of the mixed-precision kernels (mixed.cu, compiled with --fmad=false).
#pragma once

#include <cuda_runtime.h>

#include "chx_internal.cuh"

namespace chx {

// Double-float constants of the right-hand side stencil: (hi, lo) pairs.
struct FFConst {
  float2 rho, kap, gl, k1, k2;
};

// Splits a double into a (hi, lo) float pair on the host.
inline float2 split_ff(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

template <typename T>
struct DirView;

// All launchers take G / Z simulations of the group (blockIdx.z); see chgroup.cuh for layouts.
// glff[z] = gamma_z / dx^2 and aff[z] = a_z as double-float pairs, per slot.
void launch_ch_rhs_ff(const double* cn, const double* cp, float* rhi, float* rlo, double* cbar, int nx, int ny, int G,
                      const FFConst& k, const float2* glff, const double* noise, double nkx, double nky,
                      cudaStream_t st);
void launch_resid_ff(const float* fhi, const float* flo, const float* y1, const float* t1, float* x0, float* rho,
                     int ld, int nsys, int n, const DirView<float>& D, const float2* aff, int Z, size_t fz, size_t ybz,
                     cudaStream_t st);
// Reduced (cyclic-coupling) system of the first solve in double-float; grid over
// nsys systems and Z simulations (tau and yb at + z * ybz).
void launch_reduced_ff(const float* yb, const DirView<float>& D, float* tau, int nsys, size_t ybz, int Z,
                       cudaStream_t st);
// xfinish / update: y1 is the corrected first solution x0, (y2, t2) the correction solve.
void launch_ch_xfinish_ff(const float* y1, const float* t1, const float* y2, const float* t2, const DirView<float>& D,
                          float* whi, float* wlo, int nx, int ny, int G, cudaStream_t st);
void launch_ch_update_ff(const float* y1, const float* t1, const float* y2, const float* t2, const DirView<float>& D,
                         double* cn, double* cp, int nx, int ny, int G, int keep_roles, cudaStream_t st);
// Fused FP32 + refinement solves of the ADI step (one launch per direction).
// x: rows of the group (rows = G * ny), row-major f, w and the x0 scratch.
// y: columns of every simulation, then the update of cn / cp (keep_roles as
// in group_step).  prepare_solve_ff opts the kernels into large shared memory
// (call once per device, outside stream capture); solve_ff_fits says whether
// the strips of an nx x ny grid with px / py segments fit in shared memory.
int prepare_solve_ff();
bool solve_ff_fits(int nx, int ny, int px, int py);
int y_solve_cols(int n, int P);
void launch_x_solve_ff(const float* fhi, const float* flo, float* x0s, float* whi, float* wlo, int nx, int rows, int ny,
                       const DirView<float>& D, const float2* aff, cudaStream_t st);
void launch_y_solve_ff(const float* fhi, const float* flo, float* x0s, const double* cbar, double* cn, double* cp, int nx,
                       int ny, int G, const DirView<float>& D, const float2* aff, int keep_roles, cudaStream_t st);
void launch_penta_refine_ff(double* x, float* work, int n, int batch, const float* fac32, const float2* coef_ff,
                            const float* s32, cudaStream_t st);

}  // namespace chx
