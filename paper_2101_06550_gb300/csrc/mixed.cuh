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

// Fused FP32 + refinement step of the ADI scheme (launch_step_ff and the
// ensemble's phase kernels, chgroup.cuh).  prepare_solve_ff opts the kernels
// into large shared memory (once per device, outside stream capture);
// solve_ff_fits says whether the x / y strips of an nx x ny grid with px / py
// segments fit in shared memory.
int prepare_solve_ff();
bool solve_ff_fits(int nx, int ny, int px, int py);
// Points per block the fused solves aim at by default (x rows / y columns per
// block from x_solve_rows / y_solve_cols, chgroup.cuh).
constexpr int kFFTarget = 4096;
void launch_penta_refine_ff(double* x, float* work, int n, int batch, const float* fac32, const float2* coef_ff,
                            const float* s32, cudaStream_t st);

}  // namespace chx
