/*
 * chx: GB300-native (sm_103a) semi-implicit ADI stepping of the periodic 2D
 * Cahn-Hilliard equation  c_t = Lap(c^3 - c - gamma Lap c)  and the batched
 * cyclic band solvers it is built from (Gloster, arXiv 2101.06550).
 *
 * Conventions (all entry points):
 *  - Every function returns an int status: CHX_OK (0) or a negative CHX_E*
 *    code; chx_status_string() names it and chx_last_error() gives the detail
 *    of the most recent failure on the calling host thread.
 *  - Device pointers are owned by the caller.  Plans own what their
 *    *_create / *_factor call allocated (factors, small scratch) and the few
 *    lazily made buffers a function's comment names (observables scratch, an
 *    ensemble group's deviates); nothing else in this library allocates device
 *    memory.
 *  - A plan (and an ensemble) is used by one host thread at a time: calls on
 *    the same plan from several threads must be serialised by the caller.
 *    Different plans are independent.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously on it.  Errors found on the device are
 *    reported by the next chx_sync_status(plan).
 *  - Fields are row-major, v(i, j) = v[j * ld + i], i the x index.  Batched
 *    solver data is interleaved: element i of system s is at x[i * batch + s].
 *  - Only one precision per plan.  dtype CHX_F64 = double, CHX_F32 = float.
 */
#ifndef CHX_H
#define CHX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CHX_OK = 0,
  CHX_EINVAL = -1,       /* bad argument (null pointer, size out of range, mode)  */
  CHX_ESINGULAR = -2,    /* zero or tiny pivot in LU without pivoting, or a tiny
                            Sherman-Morrison / bordering denominator               */
  CHX_ENONFINITE = -3,   /* a diagnostic reduction met NaN or Inf                  */
  CHX_ENOMEM = -4,       /* a plan allocation failed                               */
  CHX_ECUDA = -5,        /* a CUDA runtime call or kernel launch failed            */
  CHX_ETIMEOUT = -6,     /* a bounded device-side wait ran out                     */
  CHX_EUNSUPPORTED = -7  /* valid request this build does not implement           */
};

enum { CHX_F64 = 0, CHX_F32 = 1 };

/* Coefficient modes of the band solvers (Secs. 4.2.4, 5.2, 5.4):
 * UNIFORM    - one value per diagonal for every row and system (cuPentUniformBatch);
 *              a..e (or a..c) each point to ONE host double.
 * SHARED     - one LHS for all systems, coefficients vary by row
 *              (cuPentConstantBatch / cuThomasConstantBatch); n host doubles each.
 * PER_SYSTEM - every system has its own LHS (cuPentBatch "Rewrite" mode);
 *              n * batch DEVICE doubles each, interleaved like the RHS.      */
enum { CHX_COEF_UNIFORM = 0, CHX_COEF_SHARED = 1, CHX_COEF_PER_SYSTEM = 2 };

enum { CHX_PREMAP_NONE = 0, CHX_PREMAP_CUBIC_MINUS_C = 1 };

/* ch_step precision: plain FP64, or FP32 sweeps with one refinement pass per
 * pentadiagonal solve whose residual, like the right-hand side, is formed in
 * double-float arithmetic (FP64 state and update).  FP32+refine keeps a step
 * within 1e-6 of max|c| of the FP64 step up to a' = (2/3) gamma dt / dx^4 of
 * about 2e4 (the 2048^2, gamma 0.005, dt 5e-4 workload).  Above a' = 5e4 the
 * solves take a second refinement pass: at a' = 3e5 a step from a rough random
 * state is then off by about 5e-6 (smooth states stay within 1e-6).
 * Its fused solves keep whole rows and column strips in shared memory: grids
 * whose rows or columns do not fit are rejected at ch_plan_create with
 * CHX_EUNSUPPORTED. */
enum { CHX_PREC_F64 = 0, CHX_PREC_F32_REFINE = 1 };

typedef struct chx_penta_plan chx_penta_plan;
typedef struct chx_tri_plan chx_tri_plan;
typedef struct chx_ch_plan chx_ch_plan;
typedef struct chx_ens chx_ens;
typedef struct chx_ch1d_plan chx_ch1d_plan;
typedef struct chx_cn1d_plan chx_cn1d_plan;

const char* chx_status_string(int status);
/* Detail of the last failure on this host thread ("" if none). */
const char* chx_last_error(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int chx_version(void);

/*
 * General 2D stencil apply (cuSten Compute 2D XY, Sec. 3.3; weights indexed
 * from the top-left of the box, i fastest, then row by row in j, Sec. 3.5.2):
 *   out(i,j) = sum_{dj=-top..bottom} sum_{di=-left..right}
 *              w[(dj+top)*(left+right+1) + (di+left)] * p(in(i+di, j+dj)),
 * p = identity, or p(c) = c^3 - c for CHX_PREMAP_CUBIC_MINUS_C (the
 * function-pointer form used for the nonlinear Cahn-Hilliard term, Sec. 3.5.2).
 *  in, out   device arrays of dtype, row-major with leading dimension ldx >= nx;
 *            out must not alias in (the blocks overlap, Sec. 3.2).
 *  w_host    HOST array of (top+bottom+1)*(left+right+1) doubles, copied into
 *            the launch; left, right, top, bottom each in [0, 7].
 *  periodic  1: wrap in both directions.  0: only points whose whole box lies
 *            inside the grid are written; the boundary cells are left untouched
 *            for the caller's own boundary conditions (Sec. 3.3).
 * Errors: CHX_EINVAL for null pointers, nx or ny < 1, ldx < nx, box out of range,
 * aliasing in/out, unknown dtype or premap; CHX_ECUDA if the launch fails.
 */
int stencil_apply_2d(const void* in, void* out, int nx, int ny, int ldx, const double* w_host, int left,
                     int right, int top, int bottom, int premap, int periodic, int dtype, void* stream);

/*
 * Batched cyclic pentadiagonal solver (Secs. 4.2.2-4.2.5 and 5.4).  Row i of
 * every system: a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1} + e_i x_{i+2}
 * = f_i, indices mod n (eq:matrix_sys1), n >= 5.  The periodic corners are
 * removed by Navon's bordering of the last two unknowns (Eqs. solve and
 * first_two) and the rest is LU without pivoting, which the paper requires to
 * be applied only to symmetric positive definite or diagonally dominant
 * matrices.  Factorisation is split from the solve (Sec. 4.2.5).
 *
 * penta_cyclic_factor: creates *plan for systems of size n.  For UNIFORM and
 *   SHARED the factors (and the bordering vectors and 2x2 tail inverse, which
 *   the paper precomputes once) are formed on the host in FP64 and uploaded;
 *   for PER_SYSTEM they are formed on the device, one thread per system, into
 *   plan-owned storage of about 9 * n * batch values, enqueued on `stream`.
 *   `batch` is the largest batch later solves may use.  dtype is the storage
 *   and sweep precision of the right-hand sides (CHX_F64 or CHX_F32).
 *   Errors: CHX_EINVAL, CHX_ESINGULAR (host factorisation met a pivot with
 *   |alpha| <= 1e3 * eps * row scale, or a tiny tail determinant), CHX_ENOMEM,
 *   CHX_ECUDA.  A singular PER_SYSTEM factorisation is flagged on the device
 *   and returned by chx_sync_status.
 * penta_cyclic_refactor: PER_SYSTEM plans only; recompute the factors from new
 *   device coefficients in the existing storage (the "Rewrite" mode, no
 *   allocation).
 * penta_cyclic_solve_batched: solves in place.  rhs_inout is a device array of
 *   n * batch values of the plan's dtype, interleaved; on return it holds x.
 *   refine = 1 (CHX_F64 plans only): the sweeps run in FP32 and one
 *   iterative-refinement pass with an FP64 residual f - A x corrects the result
 *   (uses plan-owned FP32 scratch of n * batch values).
 *   Errors: CHX_EINVAL (batch < 1 or above the plan's batch, PER_SYSTEM batch
 *   different from the factor batch, refine on an FP32 plan), CHX_ECUDA.
 */
int penta_cyclic_factor(chx_penta_plan** plan, int n, int coef_mode, const double* a, const double* b,
                        const double* c, const double* d, const double* e, int batch, int dtype, void* stream);
int penta_cyclic_refactor(chx_penta_plan* plan, const double* a, const double* b, const double* c,
                          const double* d, const double* e, void* stream);
int penta_cyclic_solve_batched(chx_penta_plan* plan, void* rhs_inout, int batch, int refine, void* stream);

/*
 * Batched cyclic tridiagonal solver (Sec. 5.3): Thomas algorithm with
 * pre-factorisation; the corners are removed with the Sherman-Morrison formula
 * x = y - (v.y)/(1 + v.z) z, with u = (-b_1, 0.., c_N), v = (1, 0.., -a_1/b_1)
 * and z = A'^{-1} u formed once at factor time.  Row i: a_i x_{i-1} + b_i x_i +
 * c_i x_{i+1} = f_i, indices mod n, n >= 3.  Modes, layouts, ownership and
 * errors as for the pentadiagonal solver (no refine option).
 */
int tri_cyclic_factor(chx_tri_plan** plan, int n, int coef_mode, const double* a, const double* b,
                      const double* c, int batch, int dtype, void* stream);
int tri_cyclic_refactor(chx_tri_plan* plan, const double* a, const double* b, const double* c, void* stream);
int tri_cyclic_solve_batched(chx_tri_plan* plan, void* rhs_inout, int batch, void* stream);

/*
 * One semi-implicit ADI step of the periodic 2D Cahn-Hilliard equation with
 * D = 1 (Eq. 3.1, eq3:ch_adi, Sec. 3.5.1):
 *   Cbar = 2 C^n - C^{n-1}
 *   r    = -(2/3)(C^n - C^{n-1}) - (2/3) gamma dt Lap_h^2 Cbar + (2/3) dt Lap_h (C^3 - C)^n
 *   (I + (2/3) gamma dt d_xxxx) w = r    (rows),
 *   (I + (2/3) gamma dt d_yyyy) v = w    (columns),
 *   C^{n+1} = Cbar + v,
 * on [0, lx) x [0, ly) with dx = lx/nx, dy = ly/ny; Lap_h is the 5-point
 * Laplacian and Lap_h^2 the 13-point biharmonic.  The first step uses
 * C^{-1} = C^0: the caller sets c_prev = c_now = c0 (Sec. 3.5.1).
 *
 * ch_plan_create: nx, ny in [8, 16384]; lx, ly, dt > 0; gamma >= 0;
 *   precision CHX_PREC_F64 or CHX_PREC_F32_REFINE.  Factors the two implicit
 *   operators on the host in FP64 and uploads them (plan-owned).
 * ch_work_bytes: size of the caller-provided device scratch `work` for ch_step
 *   (FP64: about 32 B per grid point, for r, w, Cbar and M; FP32+refine: about
 *   28 B per point; plus the reduced systems' few values per segment).
 * ch_step: advances nsteps >= 0 steps.  c_now and c_prev are device arrays of
 *   nx * ny doubles (row-major, ld = nx) that keep their roles: on return
 *   c_now = C^{n+nsteps} and c_prev = C^{n+nsteps-1}.  work must hold at
 *   least ch_work_bytes(plan) bytes, 256-byte aligned, and must not overlap
 *   the fields.  A call that repeats the previous call's three pointers, or
 *   runs four or more steps, replays CUDA graphs captured for those pointers
 *   (two steps, and one role-keeping step); the first such call captures them.
 *   While per-kernel profiling is on (ch_profile) the kernels launch one by
 *   one instead.  Errors: CHX_EINVAL, CHX_ECUDA.
 * ch_diagnostics: mass = sum c dx dy and free energy
 *   F_h = sum [ (1/4)(c^2-1)^2 + (gamma/2)(|D+x c|^2 + |D+y c|^2) ] dx dy
 *   (forward differences, periodic; Sec. 2.4 with the bulk density read as
 *   (1/4)(c^2-1)^2, the one whose derivative is c^3 - c).  mass_out and
 *   energy_out are DEVICE pointers to one double each, written asynchronously
 *   in a fixed summation order (bit-reproducible).  If c holds NaN or Inf, the
 *   plan's status becomes CHX_ENONFINITE (read it with chx_sync_status).
 */
int ch_plan_create(chx_ch_plan** plan, int nx, int ny, double lx, double ly, double gamma, double dt,
                   int precision);
size_t ch_work_bytes(const chx_ch_plan* plan);
int ch_step(chx_ch_plan* plan, double* c_now, double* c_prev, void* work, int nsteps, void* stream);
/*
 * ch_step_host: ch_step on fields that live in HOST memory.  Enqueues on
 *   `stream` the copies of h_now and h_prev (nx * ny doubles each) into the
 *   caller's device fields d_now and d_prev, nsteps steps, and the copy of the
 *   new C^n back into h_out; returns without waiting.  Host buffers should be
 *   page-locked for the copies to run asynchronously; they must stay valid
 *   until the stream reaches the copies.  Device-side arguments and errors as
 *   for ch_step.
 */
int ch_step_host(chx_ch_plan* plan, const double* h_now, const double* h_prev, double* h_out, double* d_now,
                 double* d_prev, void* work, int nsteps, void* stream);
int ch_diagnostics(chx_ch_plan* plan, const double* c, double* mass_out, double* energy_out, void* stream);

/*
 * Cahn-Hilliard-Cook equation (Sec. 7.7): the Cahn-Hilliard equation with the
 * conserved thermal forcing eta, C_t = Lap(C^3 - C - gamma Lap C) + eta, with
 *   eta_ij = sqrt(sigma / (dx dy dt)) div_h rho_ij,
 *   div_h rho_ij = (rho^x_ij - rho^x_{i-1,j}) / dx + (rho^y_ij - rho^y_{i,j-1}) / dy
 * (periodic; the backward difference makes <eta eta'> = sigma/(dx dy dt) times
 * minus the 5-point Laplacian of a Kronecker delta, the discrete form of the
 * paper's correlation), rho a 2-vector field of N(0, 1) deviates drawn afresh
 * every step.  In the ADI step of ch_step eta enters r with the weight (2/3) dt
 * of the explicit terms.  Both precisions: CHX_PREC_F32_REFINE plans form
 * the forcing term in FP64 and add it to their double-float right-hand side.
 *
 * ch_noise_normals: writes the deviates of step `step` of simulation `sim`
 *   into the device array rho (2 nx ny doubles: rho^x then rho^y, row-major,
 *   ld = nx).  Points 2b and 2b+1 take the four words of Philox4x64-10 (Salmon
 *   et al., SC 2011) with counter (b, step, 0, 0) and key (seed, sim); word w
 *   gives u = (floor(w / 2^41) + 1/2) 2^-23 and the pairs (u0, u1), (u2, u3)
 *   give (rho^x, rho^y) = sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub) (Box-Muller,
 *   evaluated in FP32 and stored as FP64).  Errors: CHX_EINVAL, CHX_ECUDA.
 * ch_step_noise: one step with caller-given deviates rho (device, 2 nx ny
 *   doubles, layout as above); c_now/c_prev keep their roles as in ch_step.
 * ch_cook_run: nsteps steps, step k drawing the deviates of step step0 + k into
 *   the caller's device scratch rho (2 nx ny doubles; FP64 plans with even nx
 *   draw them inside the right-hand-side pass, the others first with the
 *   deviate kernel: rho ends up with the same values either way).  Pairs
 *   of steps replay a captured graph whose deviates read their step index
 *   from a device counter; the first such call allocates that 8-byte counter
 *   and captures the graph (again when the pointers, sigma, seed or sim change).
 * sigma >= 0 (the paper uses 1e-14 with C = 0 initially).  rho must not overlap
 * c_now, c_prev or work.  Errors: CHX_EINVAL, CHX_ECUDA.
 */
int ch_noise_normals(double* rho, int nx, int ny, uint64_t seed, uint64_t sim, uint64_t step, void* stream);
int ch_step_noise(chx_ch_plan* plan, double* c_now, double* c_prev, void* work, const double* rho, double sigma,
                  void* stream);
int ch_cook_run(chx_ch_plan* plan, double* c_now, double* c_prev, void* work, double* rho, int nsteps,
                double sigma, uint64_t seed, uint64_t sim, uint64_t step0, void* stream);

/*
 * Coarsening observables (Secs. 2.4, 3.5.4, 7.2.3).  For a field C:
 *   out[0] mass = sum C dx dy,
 *   out[1] F_h  (as ch_diagnostics),
 *   out[2] s    = 1 / (1 - <C^2>), <.> the composite Simpson average with the
 *               periodic closure f(L) = f(0) (weights (2, 4, 2, 4, ...)/3 per
 *               direction for an even point count; the trapezoid rule, i.e. the
 *               plain mean, for an odd one),
 *   out[3] k1   = sum |C^(k)|^2 / sum |k|^-1 |C^(k)|^2 over the discrete Fourier
 *               modes k = (2 pi mx / lx, 2 pi my / ly) != 0 (the mean mode has no
 *               length scale and is left out of both sums).
 * ch_observables: one field of the plan's grid; out is a DEVICE array of 4
 *   doubles written asynchronously on `stream`.  The first call allocates
 *   plan-owned scratch (a cuFFT real-to-complex plan and ny (nx/2+1) complex
 *   values); later calls allocate nothing.
 * ens_group_observables: every active slot of a group at once, out = DEVICE
 *   array of 4 * active doubles (slot-major).  with_k1 = 0 leaves out[4s+3]
 *   NaN and needs only a small partial-sum buffer; with_k1 = 1 forms k1 with
 *   one batched real-to-complex cuFFT plan over the active slots, whose
 *   spectra (active * ny (nx/2+1) complex values) and cuFFT work area are
 *   allocated on the first such call and again when the active count changes
 *   (not counted against the ensemble's budget).
 * Both flag NaN/Inf in the field as CHX_ENONFINITE (read with chx_sync_status).
 * Errors: CHX_EINVAL, CHX_ENOMEM, CHX_ECUDA.
 *
 * chx_coarsening_rate: HOST arrays.  beta_k = -(t_k / F_k) dF/dt(t_k) (Eq.
 *   eq7:betaN; the thesis extracts dF/dt numerically, Sec. 7.3.2) for a sampled
 *   series, dF/dt from the derivative of the quadratic through three
 *   neighbouring samples: centred inside, one-sided at the ends (second order
 *   on uneven spacing).  count >= 3, t strictly increasing, F finite and
 *   non-zero, else CHX_EINVAL.
 */
int ch_observables(chx_ch_plan* plan, const double* c, double* out, void* stream);
int ens_group_observables(chx_ens* ens, int group_id, int with_k1, double* out, void* stream);
int chx_coarsening_rate(const double* t, const double* F, int count, double* beta);

/*
 * Batched 1D Cahn-Hilliard (Sec. 6.2.1, eq6:1Dnumerical): for every simulation s
 * of an interleaved batch c[i * batch + s] (i = 0..n-1, periodic on [0, l)),
 *   (I + sigma delta^4) C^{n+1} = C^n + alpha delta^2 (C^3 - C)^n,
 *   sigma = gamma dt / dx^4, alpha = dt / dx^2, dx = l / n
 * (the printed f_i lacks C_i^n; eq6:1Dnumerical has it).  The cyclic
 * pentadiagonal operator is factorised once on the host (FP64, Navon bordering
 * + LU without pivoting) by ch1d_plan_create (n >= 8, batch >= 1, l, dt > 0,
 * gamma >= 0; the plan owns about 9 n doubles of device memory).  ch1d_step
 * advances nsteps >= 0 steps in place on the device array c (n * batch
 * doubles, caller-owned, FP64); it needs no scratch.  Errors: CHX_EINVAL,
 * CHX_ESINGULAR (factorisation), CHX_ENOMEM, CHX_ECUDA.
 */
int ch1d_plan_create(chx_ch1d_plan** plan, int n, int batch, double l, double gamma, double dt);
int ch1d_step(chx_ch1d_plan* plan, double* c, int nsteps, void* stream);

/*
 * Batched Crank-Nicolson steps of the paper's two 1D periodic benchmark
 * problems, for every system s of an interleaved batch c[i * batch + s]
 * (i = 0..n-1, dx = l / n):
 *  order 4, hyperdiffusion C_t = -kappa C_xxxx (Sec. 4.2.1, eq:1d_hyper_scheme;
 *    kappa = gamma D), sigma = kappa dt / (2 dx^4):
 *    (sigma, -4 sigma, 1 + 6 sigma, -4 sigma, sigma) C^{n+1}
 *      = (-sigma, 4 sigma, 1 - 6 sigma, 4 sigma, -sigma) C^n;
 *  order 2, diffusion C_t = kappa C_xx (Sec. 5.3.2, eq5:1ddiffscheme),
 *    sigma = kappa dt / (2 dx^2):
 *    (-sigma, 1 + 2 sigma, -sigma) C^{n+1} = (sigma, 1 - 2 sigma, sigma) C^n.
 * In both the explicit row is twice the identity minus the implicit one
 * (B = 2I - A), so a step is C^{n+1} = 2 A^{-1} C^n - C^n: one cyclic
 * pentadiagonal (Navon bordering + LU) or tridiagonal (Thomas + Sherman-
 * Morrison) solve with right-hand side C^n and no explicit half to form.
 * cn1d_plan_create: order 2 or 4; n >= 6 (order 4) or >= 3 (order 2);
 * batch >= 1; l, dt > 0; kappa >= 0.  Every plan owns n * batch doubles of
 * sweep scratch.  rewrite selects the paper's benchmark variant (Sec. 4.3):
 *   0 (Constant)  the matrix is factorised once on the host in FP64; the plan
 *                 also owns about 9 n doubles of factors;
 *   1 (Rewrite)   the plan owns (order + 1) * n * batch doubles of per-system
 *                 matrix entries plus a PER_SYSTEM solver plan (about 9 n batch
 *                 doubles of factors), and every step resets the entries and
 *                 refactorises every system on the device before the sweep.
 * cn1d_step advances nsteps >= 0 steps in place on the caller-owned device
 * array c (n * batch doubles).  Errors: CHX_EINVAL,
 * CHX_ESINGULAR (host factorisation; a Rewrite plan's device factorisation
 * reports it through chx_sync_status), CHX_ENOMEM, CHX_ECUDA.
 */
int cn1d_plan_create(chx_cn1d_plan** plan, int order, int n, int batch, double l, double kappa, double dt,
                     int rewrite);
int cn1d_step(chx_cn1d_plan* plan, double* c, int nsteps, void* stream);

/*
 * Ensemble runtime: many simulations of uneven sizes advanced together (the
 * batches of 2D simulations per domain size behind the thesis's statistics,
 * Sec. 7.3.2, and its note that batches of different sizes want one LHS per
 * distinct matrix, Sec. 8).  Every simulation is the ADI step of ch_step with
 * the ensemble's dt and precision on an n x n grid of side l.
 *  - A group holds simulations with the same (n, l): packed device-resident
 *    state (C^n, C^{n-1}) for `capacity` slots, per-slot LHS factors (so the
 *    slots may have different gamma), and one set of batched launches per step.
 *    Device memory is allocated only by ens_create, ens_group_create and the
 *    first ens_group_set_cook / ens_group_observables of a group; ens_group_create fails with CHX_ENOMEM when the
 *    group would take the ensemble past hbm_budget_bytes (0 = no budget).
 *  - Slots [0, active) of each group are stepped (ens_group_set_active); the
 *    caller keeps active simulations packed with ens_slot_move.  A simulation's
 *    arithmetic does not depend on which other slots are active.
 *  - ens_step advances every active slot of every group by nsteps, replaying a
 *    CUDA graph that holds two steps of all groups (one graph branch per
 *    group); the graph is rebuilt after any change of groups or active counts.
 *  - ens_slot_load sets C^n = c0 and C^{n-1} = cm1 (or c0 if cm1 is NULL) for a
 *    slot and, if gamma >= 0 differs from the slot's, refactorises the slot's
 *    operators for it (host FP64, synchronous); ens_slot_read copies C^n (and
 *    optionally C^{n-1}) out.  ens_slot_move copies state and factors.  Pointers may
 *    be host or device memory (cudaMemcpyDefault); n*n doubles each.
 *  - ens_autotune times `trial` steps per candidate segment count of a group's
 *    partitioned sweeps and keeps the fastest: every candidate x count with the
 *    y count held, then every y count with the chosen x count (the two are
 *    independent; px_out / py_out receive them).  The simulations' state is
 *    saved and restored, so the call changes no result other than by rounding
 *    order.
 *  - ens_group_set_cook turns on the Cahn-Hilliard-Cook forcing of ch_cook_run
 *    (Sec. 7.7) for every slot of a group (either precision): each later step
 *    of the group first draws the deviates of slot s with simulation id s, key
 *    seed, at the group's step counter
 *    (starting at step0 and advanced on the device, so graph replays draw
 *    fresh deviates), then takes the forced step.  It allocates the group's
 *    deviate scratch (2 capacity n^2 doubles, counted against the budget) on
 *    first use and synchronises the device; sigma = 0 turns the forcing off
 *    and frees the scratch.
 * Destroy with chx_plan_destroy; chx_sync_status works on the ensemble too.
 * Errors: CHX_EINVAL (bad ids, sizes, slots), CHX_ENOMEM, CHX_ECUDA.
 */
int ens_create(chx_ens** ens, int precision, double dt, size_t hbm_budget_bytes);
int ens_group_create(chx_ens* ens, int n, double l, double gamma, int capacity, int* group_id);
int ens_group_destroy(chx_ens* ens, int group_id);
int ens_group_set_active(chx_ens* ens, int group_id, int active);
int ens_group_set_cook(chx_ens* ens, int group_id, double sigma, uint64_t seed, uint64_t step0);
int ens_slot_load(chx_ens* ens, int group_id, int slot, const double* c0, const double* cm1, double gamma,
                  void* stream);
int ens_slot_read(chx_ens* ens, int group_id, int slot, double* c_now, double* c_prev, void* stream);
int ens_slot_move(chx_ens* ens, int group_id, int from, int to, void* stream);
int ens_step(chx_ens* ens, int nsteps, void* stream);
int ens_group_step(chx_ens* ens, int group_id, int nsteps, void* stream);
int ens_autotune(chx_ens* ens, int group_id, int trial, int* px_out, int* py_out, void* stream);
int ens_info(chx_ens* ens, int group_id, int* n, int* capacity, int* active, int* px, int* py, size_t* bytes);
/* FP32 + refinement ensembles step every group with three launches per step,
 * one per phase (right-hand side, x solves, y solves with the update): each a
 * persistent grid whose blocks stride over the work items of all groups, packed
 * group after group (the thesis's batches of uneven 2D simulations, Sec. 7.3.2,
 * with one LHS per distinct matrix, Sec. 8); every group keeps tiles of its own
 * shape.  ens_tune_schedule times `trial` steps for each candidate schedule --
 * group order (0: most work per item first, 1: least first), points per work
 * item of the solves (2048, 4096 or 8192; each group's x rows and y columns per
 * item follow) and the y phase's blocks per SM -- keeps the fastest, and
 * reports the order, the points per item and the blocks of the three phases
 * (blocks_out: 3 ints; any output may be NULL).
 * It saves C^{n-1} of the active slots and puts it back, so no simulation
 * changes; the saved copy counts against the HBM budget (CHX_ENOMEM).
 * ens_schedule_info reports the current layout (items_out, blocks_out: 3 ints).
 * Both return CHX_EUNSUPPORTED for FP64 ensembles and, for the tuner, when no
 * group is active or more than 256 groups are. */
int ens_tune_schedule(chx_ens* ens, int trial, int* order_out, int* target_out, int* blocks_out, void* stream);
int ens_schedule_info(chx_ens* ens, int* items_out, int* blocks_out, int* target_out, int* order_out);
size_t ens_bytes_used(const chx_ens* ens);

/*
 * Allocation-free mass / free-energy reduction.  The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc (code running
 * where the device allocator may not be used, or hosts that reserve all device
 * memory up front), so it needs no plan and allocates nothing.  It computes the
 * same two sums as ch_diagnostics (same definitions; the summation order
 * differs, by rows), for a row-major nx x ny field c on [0,lx) x [0,ly).
 *  c, mass_out, energy_out  device pointers (one double each for the outputs),
 *                           written asynchronously on `stream`.
 *  Scratch: one partial-sum triple per row in a fixed device array of 16384
 *  rows (384 KiB) that every GPU loading this library holds until exit; ny above
 *  16384 is rejected with CHX_EINVAL.  All calls share that array and it keeps
 *  the last call's contents (each call overwrites every row it reads, so nothing
 *  needs clearing); calls that overlap on the GPU (different streams, or
 *  different host threads) race on it and must be serialised by the caller.
 *  The first call on each device looks up the array's device address
 *  (cudaGetSymbolAddress) with that device current; make that first call
 *  before any stream capture.
 *  A NaN or Inf in c makes both outputs NaN.
 * Errors: CHX_EINVAL (null pointer, nx or ny < 1, ny > 16384, lx or ly <= 0,
 * gamma < 0), CHX_ECUDA.
 */
int ch_diagnostics_noalloc(const double* c, int nx, int ny, double lx, double ly, double gamma, double* mass_out,
                           double* energy_out, void* stream);

/* Profiling aid.  ch_profile(plan, 1) makes every later ch_step bracket each
 * kernel it launches with CUDA events on the launch stream (a few microseconds
 * of host time per launch); ch_profile(plan, 0) stops it.  ch_profile_read
 * waits for the recorded events, adds their elapsed times to per-kernel
 * totals, copies up to max_slots totals (milliseconds) and launch counts into
 * ms[] and launches[] (either may be NULL), optionally resets them, and returns
 * the number of kernel slots (or a negative status).  ch_profile_slot_name
 * names a slot ("" if out of range). */
int ch_profile(chx_ch_plan* plan, int enable);
int ch_profile_read(chx_ch_plan* plan, double* ms, long long* launches, int max_slots, int reset);
const char* ch_profile_slot_name(int slot);

/* Measurement aid (no counterpart in the paper): the device's sustained FP64
 * fused multiply-add rate, for the roofline of the FP64 kernels, which are
 * bound by the FP64 pipe rather than by HBM.  Runs a throughput kernel of
 * independent DFMA chains over every SM in two operand forms (constants as
 * kernel parameters, and loaded into registers; each one warm-up launch, then
 * two timed ones, CUDA events on `stream`) and writes the larger rate, in 1e9
 * DFMA per second, to *gops_out (host pointer): some forms of the same chains
 * issue at a lower rate.  Synchronous; allocates and frees a 24-byte device
 * scratch.  Returns CHX_EINVAL for a NULL pointer, CHX_ECUDA on a CUDA error. */
int chx_fp64_fma_rate(double* gops_out, void* stream);

/* Waits for the plan's last stream and returns (and clears) the first error the
 * device recorded for this plan, or CHX_OK.  Works for every plan type. */
int chx_sync_status(void* plan);
/* Frees a plan of any type (NULL is allowed).  The caller must make sure no
 * work using the plan is still in flight. */
void chx_plan_destroy(void* plan);

#ifdef __cplusplus
}
#endif

#endif /* CHX_H */
