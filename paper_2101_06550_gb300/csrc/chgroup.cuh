// A group of same-shape Cahn-Hilliard simulations advanced together by one set
// of batched launches (the ADI step of Eq. 3.1 for G fields at once).  The
// single-simulation plan (ch_plan_*) is a group of one; the ensemble runtime
// (ens.cu) keeps one group per distinct (n, gamma, L, dt).
#pragma once

#include <utility>
#include <vector>

#include "chx_internal.cuh"
#include "mixed.cuh"

namespace chx {

// Partitioned (SPIKE-type) factors of the constant cyclic operator
// I + a delta^4 along one direction.  Every simulation slot of a group has its
// own block (its own gamma, hence its own a): slot z's factors start at
// z * 4m (lu, vw) and z * (4P)^2 (rinv).
struct SpikeDir {
  int n = 0, P = 1, m = 0, slots = 0;
  int band = 0;                 // reduced inverse kept for segment distances <= band (all slots)
  double* d_a = nullptr;        // slots: a = (2/3) gamma dt / h^4
  double* d_lu = nullptr;       // slots x 4m: ralpha, beta, gam, del of the segment block
  double* d_vw = nullptr;       // slots x 4m: spikes V0, V1, W0, W1
  double* d_rinv = nullptr;     // slots x (4P)^2 reduced-system inverse
  float* d_a32 = nullptr;
  float2* d_aff = nullptr;      // a as a double-float pair
  float4* d_lu4 = nullptr;      // slots x m: the FP32 factors of each row (ralpha, beta, gam, del)
  float* d_vw32 = nullptr;
  float* d_rinv32 = nullptr;
  // the FP64 spikes and reduced inverse less their FP32 roundings (v - (float)v):
  // with d_vw32 / d_rinv32 they form the double-float pairs of the first
  // mixed-precision solve's cyclic coupling
  float* d_vwlo = nullptr;
  float* d_rinvlo = nullptr;
  // the reduced inverse by block offset, for the fused mixed-precision solves:
  // rb[(d*4 + u)*4P + q] = rinv[q][4*((q/4 + d) mod P) + u], d in [0, P), so
  // that consecutive output rows q read consecutive words; high and low floats
  float* d_rb32 = nullptr;
  float* d_rblo = nullptr;
  // the four spikes of each row packed (V0, V1, W0, W1), high and low floats,
  // so the fused solves fetch a row's spikes with one 128-bit load
  float4* d_vw4 = nullptr;
  float4* d_vw4lo = nullptr;
  // rows [plo, phi) of every slot's segment block where the four spikes'
  // magnitudes sum to at most 1: the first mixed-precision solve forms x0 there
  // with plain FP32 arithmetic (exact accumulation elsewhere)
  int plo = 0, phi = 0;
  bool pset = false;
  // refinement passes of the mixed-precision solves, for the stiffest slot
  int passes = 1;
};
// Refinement passes for the operator I + a delta^4: one up to a = 5e4 (the
// 2048^2 workload's a = 1.9e4 meets 1e-6 with one), two above.  Measured at
// a = 3e5 from a rough state: 5.5e-5 of max|c| after one pass, 4.5e-6 after
// two; a third pass makes it worse (2.3e-5): the partitioned FP32 solve's
// own error on the ever smaller correction sets a floor, which a numpy model
// of the same solve reproduces.
inline int refine_passes(double a) { return a <= 5e4 ? 1 : 2; }

// Per-direction view handed to the kernels: slot of system j = blockIdx.z + j / spp.
template <typename T>
struct DirView {
  const T* a;
  const T* lu;
  const T* vw;
  const T* rinv;
  int m, P, spp, band;
  float rm;  // 1 / m, for seg_row
  const float* vwlo;    // FP32 views: low parts of vw and rinv (nullptr for FP64)
  const float* rinvlo;
  const float* rb;      // FP32 views: rinv by block offset, high and low floats
  const float* rblo;
  const float4* vw4;    // FP32 views: packed spikes per row, high and low floats
  const float4* vw4lo;
  int plo, phi;         // FP32 views: rows of plain FP32 spike correction (SpikeDir)
  const float4* lu4;    // FP32 views: factors packed per row (SpikeDir::d_lu4; lu is unused)
};

// Segment s and row r of global row i for segments of m rows, without an
// integer division: a float reciprocal estimate, then one correction step
// (the estimate is off by at most one for i < 2^22).
__device__ __forceinline__ void seg_row(int i, int m, float rm, int& s, int& r) {
  s = (int)((float)i * rm);
  r = i - s * m;
  if (r < 0) {
    --s;
    r += m;
  } else if (r >= m) {
    ++s;
    r -= m;
  }
}

struct ChGroup;

// One group's fused FP32 + refinement step (mixed.cu): everything its three
// launches need, passed by value to a single plan's kernels and as a device
// array to the ensemble's phase kernels.  The fields of slot z are at
// st[b] + z * nx * ny; at step parity q, C^n is in st[cur0 ^ q] and C^{n-1}
// (overwritten by C^{n+1}) in the other buffer.
struct FFStep {
  int nx, ny, G;       // grid and simulations stepped
  int iso;             // square cells (rho = 1): the exact-scaling Laplacian
  int tx, ty;          // right-hand-side tiles per simulation along x and y
  int xs;             // x solve: rows per block
  int ysc, ynt, ypad;  // y solve: columns per block (1 to 32), threads per block (512 or 1024), shared-memory pad
  int yrb;             // y solve: the slot's reduced inverse staged in shared memory (single plans, when it fits)
  int xpass, ypass;    // refinement passes of the x / y solve (SpikeDir::passes)
  int lgx, lgy;        // log2 of the segment lengths (-1 if not a power of two)
  FFConst k;
  const float2* glff;  // per slot gamma / dx^2 (double-float)
  const double* noise; // Cahn-Hilliard-Cook deviates (nullptr: none)
  double nkx, nky;
  DirView<float> X, Y;
  const float2* affX;  // per slot a' along x and y (double-float)
  const float2* affY;
  double* st[2];
  int cur0;
  float *fhi, *flo, *whi, *wlo, *x0s;  // work: right-hand side, x result, x0 scratch
  float2* cbar;                        // work: Cbar as a double-float pair
};

// Builds the parameters of the group's fused step for its first G slots, with
// cur / prev as C^n / C^{n-1} (st = {cur, prev}, cur0 = 0); the solves' blocks
// take about `target` points each.
FFStep ff_step_params(const ChGroup* g, int G, double* cur, double* prev, void* work, int target = kFFTarget,
                      bool balance = false);
// The three launches of one fused step (keep_roles as in group_step).
// Shared-memory bytes of the fused x / y solves for an n-point system with P
// segments (xs rows / S columns per block), and the tile shapes for about
// `target` points per block (0: does not fit).
size_t x_solve_smem(int n, int ny, int P, int xs);
size_t y_solve_smem(int n, int P, int S, int rbs = 0);
int x_solve_rows(int n, int ny, int P, int target);
int y_solve_cols(int n, int P, int target);
// The y strips of a single plan's step: the width S (and 512 or 1024 threads)
// that puts the fewest columns on the busiest SM, from the default width and
// every even width up to 32 (a width that fits one block per SM takes 1024
// threads); rbs: whether the reduced inverse also fits in shared memory at the
// same blocks per SM.  Without balance: the default width, 512 threads, no staging.
void y_solve_shape(int nx, int ny, int G, int P, int target, bool balance, int* S, int* nt, int* rbs);
int y_solve_pad(int m, int S);
int log2_exact(int m);

// The ensemble's phase kernels: one launch per phase (0: right-hand side,
// 1: x solves, 2: y solves and updates) covers the work items of every group.
// Items are numbered group after group in the order `order` (device array of
// ngroups group indices into steps); start[k] is the first item of the k-th
// group of the order (ngroups + 1 entries, start[ngroups] = nitems).  Block b
// takes items b, b + blocks, ...; every group keeps its own tile shape.  smem:
// the largest of the groups' blocks (for the right-hand side phase, 0 or 1:
// whether any group has Cook forcing).
void launch_ens_phase_ff(int phase, const FFStep* steps, const int* order, const int* start, int ngroups, int nitems,
                         int blocks, int parity, size_t smem, cudaStream_t st);
// Items of one phase of a group, and the most blocks per SM its kernel can keep
// resident with `smem` bytes of dynamic shared memory.
int ens_phase_items(int phase, const FFStep& P);
int ens_phase_occupancy(int phase, size_t smem);
// Most dynamic shared memory a block of the x / y phase kernels may take (they
// keep the current group's parameters in static shared memory besides).
size_t ens_phase_smem_max();

// Per-kernel CUDA-event timing (ch_profile).
enum ProfSlot { kRhs, kLocX, kRedX, kRefX, kLoc2X, kRed2X, kFinX, kLocY, kRedY, kRefY, kLoc2Y, kRed2Y, kUpd, kRhsLap,
                kXSolve, kYSolve, kSlots };
extern const char* const kSlotName[kSlots];

struct Prof {
  int on = 0;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pend;
  std::vector<int> slot;
  double ms[kSlots] = {0};
  long long n[kSlots] = {0};
  cudaEvent_t get();
  void release_all();
  int read(double* ms_out, long long* n_out, int max_slots, int reset);
};

struct ProfScope {
  Prof* p;
  int slot;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  ProfScope(Prof* p_, int slot_, cudaStream_t st_);
  ~ProfScope();
};

struct ObsState;

// The three launches of one fused FP32 step (keep_roles as in group_step).
void launch_step_ff(const FFStep& P, int keep_roles, Prof* prof, cudaStream_t st);

struct ChGroup {
  int nx = 0, ny = 0, G = 0, precision = 0;
  double lx = 0, ly = 0, gamma = 0, dt = 0, dx = 0, dy = 0;
  double rho = 0, kap = 0, k1 = 0, k2 = 0;  // right-hand side constants shared by the slots
  FFConst kff;                               // the same as double-float pairs (gl unused there)
  double* d_gl = nullptr;                    // slots: gamma / dx^2
  // Cahn-Hilliard-Cook deviates for the next step (FP64 only; nullptr: none),
  // 2 nx ny doubles per slot, and the forcing weights (2/3) dt amp / dx, / dy
  const double* noise = nullptr;
  double nkx = 0, nky = 0;
  // ... or drawn by the FP64 right-hand side itself (group_cook_deviates): into
  // noise_w, key (noise_seed, noise_sim0 + slot), step *noise_dstep (or noise_step)
  double* noise_w = nullptr;
  uint64_t noise_seed = 0, noise_sim0 = 0, noise_step = 0;
  const uint64_t* noise_dstep = nullptr;
  struct ObsState* obs = nullptr;  // observables scratch, made on first use (obs.cu)
  float2* d_glff = nullptr;
  SpikeDir X, Y;
  // work layout (byte offsets), for G fields
  size_t off_f = 0, off_flo = 0, off_w = 0, off_wlo = 0, off_y1 = 0, off_y2 = 0, off_x0 = 0, off_cb = 0, off_m = 0;
  size_t off_ybx = 0, off_tx = 0, off_ybx2 = 0, off_tx2 = 0, off_yby = 0, off_ty = 0, off_yby2 = 0, off_ty2 = 0;
  size_t work_bytes = 0;
  size_t factor_bytes = 0;  // device bytes of the per-slot factors and parameters (group_init)
};

// Validates, factorises both directions on the host (FP64) for `gamma` and
// uploads them into every slot.  px / py > 0 force the segment counts (the
// ensemble autotuner); 0 = default.
int group_init(ChGroup* g, int nx, int ny, double lx, double ly, double gamma, double dt, int precision, int G,
               int px = 0, int py = 0);
// Refactorises slot z of the group for a new gamma (host FP64, synchronous upload).
int group_set_gamma(ChGroup* g, int z, double gamma);
// Sets up the Cahn-Hilliard-Cook deviates of the group's next step for its
// first gact slots (slot z: key (seed, sim0 + z)), into rho (2 nx ny doubles
// per slot): drawn in place by the FP64 right-hand side when nx is even,
// otherwise by the standalone deviate kernel on st first.  d_step, when given,
// holds the step index on the device.  group_cook_clear undoes it.
int group_cook_deviates(ChGroup* g, int gact, double* rho, uint64_t seed, uint64_t sim0, uint64_t step,
                        const uint64_t* d_step, cudaStream_t st);
void group_cook_clear(ChGroup* g);
// Copies slot `from`'s parameters onto slot `to` (device to device, on st).
int group_move_params(ChGroup* g, int from, int to, cudaStream_t st);
void group_free(ChGroup* g);
// Candidate segment counts for n points and nsys systems (divisors of n with
// at least 8 points per segment), default first.
std::vector<int> segment_candidates(int n, int nsys, int precision);
// One step for the first `gact` fields of the group: cur / prev point to
// gact contiguous fields of nx*ny doubles (C^n, C^{n-1}).  keep_roles = 0
// writes C^{n+1} over prev (caller swaps); 1 writes C^n into prev and C^{n+1}
// into cur.
// status: the plan's device status word (no step kernel writes it at present); may be null.
// Coarsening observables [mass, F_h, s, k1] of the first gact fields into the
// device array out (4 per field; k1 only with with_k1 and gact == 1, else NaN).
int group_observables(ChGroup* g, int gact, const double* fields, double* out, int with_k1, int* status,
                      cudaStream_t st);
void obs_free(ObsState* o);
void group_step(ChGroup* g, int gact, double* cur, double* prev, void* work, int keep_roles, cudaStream_t st,
                Prof* prof, int* status);

}  // namespace chx
