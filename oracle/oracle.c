/*
 * Plain, slow, FP64 CPU oracle for the semi-implicit ADI Cahn-Hilliard step and
 * the batched cyclic band solvers it is built from (Gloster, arXiv 2101.06550).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library; the two are compared on the same
 * seeded inputs.
 *
 * Every function follows the paper's statement of the operation, in the
 * paper's order, without blocking, fusion or reordering:
 *   - cyclic pentadiagonal solve: Navon's bordering of the last two unknowns
 *     (Sec. 4.2.2, Eqs. xhat, solve, first_two) on top of the pentadiagonal LU
 *     without pivoting (Sec. 4.2.3, factor / forward / back steps);
 *   - cyclic tridiagonal solve: Thomas pre-factorisation and sweeps (Sec. 5.3.1)
 *     with the Sherman-Morrison correction for the corners (Sec. 5.3.3);
 *   - general 2D stencil apply with periodic or non-periodic boundaries
 *     (Sec. 3.3, weights indexed from the top-left, i fastest, row by row in j);
 *   - the ADI step of Eq. 3.1 (eq3:ch_adi) with C-bar = 2C^n - C^{n-1},
 *     the 13-point biharmonic and the 5-point Laplacian (Sec. 3.5.1-3.5.2);
 *   - mass and free energy of a field (Sec. 2.4, eq2:dFdt_ch).
 * Readings of garbled or silent passages are listed where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ESINGULAR -2
#define ORC_ENOMEM -3

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

/* ---------------------------------------------------------------------------
 * Pentadiagonal LU without pivoting of an m x m band matrix (Sec. 4.2.3).
 * Row r of the band: a[r] x_{r-2} + b[r] x_{r-1} + c[r] x_r + d[r] x_{r+1}
 * + e[r] x_{r+2}; entries that fall outside the matrix are ignored.  The
 * factors are L (diagonal alpha, sub-diagonals beta and epsilon = a) and R
 * (unit diagonal, super-diagonals gamma and delta), computed in the order of
 * the paper's factorisation steps.  Pivot test: |alpha_r| must exceed
 * 1e3 * DBL_EPSILON * (|a|+|b|+|c|+|d|+|e|) of its row, else singular.
 * ------------------------------------------------------------------------- */
typedef struct {
  int m;
  double *alpha, *beta, *eps, *gam, *del;
} band_lu;

static void band_lu_free(band_lu* f) {
  free(f->alpha); free(f->beta); free(f->eps); free(f->gam); free(f->del);
}

static int band_lu_factor(int m, const double* a, const double* b, const double* c,
                          const double* d, const double* e, band_lu* f) {
  f->m = m;
  f->alpha = calloc(m, sizeof(double)); f->beta = calloc(m, sizeof(double));
  f->eps = calloc(m, sizeof(double)); f->gam = calloc(m, sizeof(double));
  f->del = calloc(m, sizeof(double));
  if (!f->alpha || !f->beta || !f->eps || !f->gam || !f->del) { band_lu_free(f); return ORC_ENOMEM; }
  for (int r = 0; r < m; ++r) {
    double ar = r >= 2 ? a[r] : 0.0, br = r >= 1 ? b[r] : 0.0;
    double dr = r + 1 < m ? d[r] : 0.0, er = r + 2 < m ? e[r] : 0.0;
    f->eps[r] = ar;
    f->beta[r] = br - (r >= 2 ? ar * f->gam[r - 2] : 0.0);
    f->alpha[r] = c[r] - (r >= 2 ? ar * f->del[r - 2] : 0.0) - (r >= 1 ? f->beta[r] * f->gam[r - 1] : 0.0);
    double scale = fabs(ar) + fabs(br) + fabs(c[r]) + fabs(dr) + fabs(er);
    if (!(fabs(f->alpha[r]) > 1e3 * 2.220446049250313e-16 * scale)) return ORC_ESINGULAR;
    f->gam[r] = (dr - (r >= 1 ? f->beta[r] * f->del[r - 1] : 0.0)) / f->alpha[r];
    f->del[r] = er / f->alpha[r];
  }
  return ORC_OK;
}

/* Solve (L R) x = f: forward for g with f = L g, back-substitute R x = g. */
static void band_lu_solve(const band_lu* f, const double* rhs, double* x) {
  int m = f->m;
  double* g = x; /* g is overwritten by x in the back sweep */
  for (int r = 0; r < m; ++r) {
    double s = rhs[r];
    if (r >= 2) s -= f->eps[r] * g[r - 2];
    if (r >= 1) s -= f->beta[r] * g[r - 1];
    g[r] = s / f->alpha[r];
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = g[r];
    if (r + 1 < m) s -= f->gam[r] * x[r + 1];
    if (r + 2 < m) s -= f->del[r] * x[r + 2];
    x[r] = s;
  }
}

/* ---------------------------------------------------------------------------
 * Cyclic pentadiagonal solve, one system (Sec. 4.2.2).
 * Row i (0-based): a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1} + e_i x_{i+2}
 * = f_i with indices mod n (eq:matrix_sys1).  Coefficients and vectors are read
 * with strides so the batched interleaved layout x[i*batch + s] can be used.
 * Bordering: the unknowns split into xhat = x_0..x_{n-3} and the tail
 * (x_{n-2}, x_{n-1}); E is A restricted to xhat, k the columns of A that couple
 * the tail into the first n-2 rows, h^T the part of the last two rows acting on
 * xhat, D the 2x2 tail block.  Then (Eq. first_two)
 *   x_tail = [D - h^T E^{-1} k]^{-1} (f_tail - h^T E^{-1} fhat)
 * and (Eq. solve) xhat = E^{-1}(fhat - k x_tail).  Requires n >= 5 so that the
 * five offsets of a row are distinct columns.
 * ------------------------------------------------------------------------- */
int oracle_penta_cyclic_solve(int n, const double* a, const double* b, const double* c,
                              const double* d, const double* e, long cs,
                              const double* f, long fs, double* x, long xs) {
  if (n < 5) return ORC_EINVAL;
  int m = n - 2;
  double *ea = malloc(5 * m * sizeof(double));
  double *k0 = calloc(m, sizeof(double)), *k1 = calloc(m, sizeof(double));
  double *fh = malloc(m * sizeof(double)), *z = malloc(m * sizeof(double));
  double *z0 = malloc(m * sizeof(double)), *z1 = malloc(m * sizeof(double));
  int rc = ORC_OK;
  band_lu lu = {0};
  if (!ea || !k0 || !k1 || !fh || !z || !z0 || !z1) { rc = ORC_ENOMEM; goto done; }
  double *eb = ea + m, *ec = ea + 2 * m, *ed = ea + 3 * m, *ee = ea + 4 * m;
  /* Split each of the first m rows into its E part and its k part. */
  for (int r = 0; r < m; ++r) {
    double co[5] = {a[r * cs], b[r * cs], c[r * cs], d[r * cs], e[r * cs]};
    double* band[5] = {&ea[r], &eb[r], &ec[r], &ed[r], &ee[r]};
    for (int o = -2; o <= 2; ++o) {
      int col = wrap(r + o, n);
      *band[o + 2] = 0.0;
      if (col < m) {
        if (col == r + o) *band[o + 2] = co[o + 2];
        else { rc = ORC_EINVAL; goto done; } /* cannot happen for n >= 5 */
      } else if (col == m) {
        k0[r] += co[o + 2];
      } else {
        k1[r] += co[o + 2];
      }
    }
    fh[r] = f[r * fs];
  }
  rc = band_lu_factor(m, ea, eb, ec, ed, ee, &lu);
  if (rc != ORC_OK) goto done;
  band_lu_solve(&lu, fh, z);   /* E^{-1} fhat */
  band_lu_solve(&lu, k0, z0);  /* E^{-1} k (first column)  */
  band_lu_solve(&lu, k1, z1);  /* E^{-1} k (second column) */
  /* Last two rows: S = D - h^T E^{-1} k, rhs = f_tail - h^T E^{-1} fhat. */
  double S[2][2], t[2];
  for (int q = 0; q < 2; ++q) {
    int r = m + q;
    double co[5] = {a[r * cs], b[r * cs], c[r * cs], d[r * cs], e[r * cs]};
    double Dq0 = 0.0, Dq1 = 0.0, hz = 0.0, hz0 = 0.0, hz1 = 0.0;
    for (int o = -2; o <= 2; ++o) {
      int col = wrap(r + o, n);
      double v = co[o + 2];
      if (col < m) { hz += v * z[col]; hz0 += v * z0[col]; hz1 += v * z1[col]; }
      else if (col == m) Dq0 += v;
      else Dq1 += v;
    }
    S[q][0] = Dq0 - hz0;
    S[q][1] = Dq1 - hz1;
    t[q] = f[r * fs] - hz;
  }
  double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
  double sc = fabs(S[0][0] * S[1][1]) + fabs(S[0][1] * S[1][0]);
  if (!(fabs(det) > 1e3 * 2.220446049250313e-16 * sc)) { rc = ORC_ESINGULAR; goto done; }
  double xt0 = (S[1][1] * t[0] - S[0][1] * t[1]) / det;
  double xt1 = (S[0][0] * t[1] - S[1][0] * t[0]) / det;
  for (int r = 0; r < m; ++r) x[r * xs] = z[r] - z0[r] * xt0 - z1[r] * xt1;
  x[m * xs] = xt0;
  x[(m + 1) * xs] = xt1;
done:
  band_lu_free(&lu);
  free(ea); free(k0); free(k1); free(fh); free(z); free(z0); free(z1);
  return rc;
}

/* Batched interleaved form: element i of system s at [i*batch + s].
 * coef_mode 0: one shared set of n coefficients per diagonal;
 * coef_mode 1: per-system coefficients, interleaved like the right-hand side. */
int oracle_penta_cyclic_batch(int n, int batch, int coef_mode, const double* a, const double* b,
                              const double* c, const double* d, const double* e,
                              const double* f, double* x) {
  for (int s = 0; s < batch; ++s) {
    long off = coef_mode ? s : 0, cs = coef_mode ? batch : 1;
    int rc = oracle_penta_cyclic_solve(n, a + off, b + off, c + off, d + off, e + off, cs,
                                       f + s, batch, x + s, batch);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Tridiagonal Thomas algorithm with pre-factorisation (Sec. 5.3.1):
 * chat_1 = c_1/b_1, chat_i = c_i/(b_i - a_i chat_{i-1});
 * dhat_1 = d_1/b_1, dhat_i = (d_i - a_i dhat_{i-1})/(b_i - a_i chat_{i-1});
 * x_N = dhat_N, x_i = dhat_i - chat_i x_{i+1}.  (The printed back sweep reads
 * "dhat_i - a_i chat_i"; the Thomas recurrence it derives from needs x_{i+1}.)
 * ------------------------------------------------------------------------- */
static int thomas(int n, const double* a, const double* b, const double* c, long cs,
                  const double* rhs, double* x, double* chat) {
  double prev_c = 0.0, prev_d = 0.0;
  for (int i = 0; i < n; ++i) {
    double ai = i > 0 ? a[i * cs] : 0.0;
    double den = b[i * cs] - ai * prev_c;
    double scale = fabs(ai) + fabs(b[i * cs]) + fabs(c[i * cs]);
    if (!(fabs(den) > 1e3 * 2.220446049250313e-16 * scale)) return ORC_ESINGULAR;
    chat[i] = (i + 1 < n ? c[i * cs] : 0.0) / den;
    x[i] = (rhs[i] - ai * prev_d) / den;
    prev_c = chat[i];
    prev_d = x[i];
  }
  for (int i = n - 2; i >= 0; --i) x[i] = x[i] - chat[i] * x[i + 1];
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Cyclic tridiagonal solve (Sec. 5.3.3).  Row i: a_i x_{i-1} + b_i x_i +
 * c_i x_{i+1} = f_i, indices mod n, so a_1 sits in the top-right corner and
 * c_N in the bottom-left.  With the paper's choice, generalised to per-row
 * coefficients: u = (-b_1, 0, ..., 0, c_N)^T, v = (1, 0, ..., 0, -a_1/b_1)^T,
 * A' = A - u v^T (so A'_11 = 2 b_1, A'_NN = b_N + a_1 c_N / b_1, no corners);
 * solve A' y = f and A' z = u, then x = y - (v.y)/(1 + v.z) z.  (The printed
 * "A'x = U" for the second solve means z.)  Requires n >= 3.
 * ------------------------------------------------------------------------- */
int oracle_tri_cyclic_solve(int n, const double* a, const double* b, const double* c, long cs,
                            const double* f, long fs, double* x, long xs) {
  if (n < 3) return ORC_EINVAL;
  double* bp = malloc(n * sizeof(double));
  double *rhs = malloc(n * sizeof(double)), *u = calloc(n, sizeof(double));
  double *y = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
  double* chat = malloc(n * sizeof(double));
  double *ap = malloc(n * sizeof(double)), *cp = malloc(n * sizeof(double));
  int rc = ORC_OK;
  if (!bp || !rhs || !u || !y || !z || !chat || !ap || !cp) { rc = ORC_ENOMEM; goto done; }
  double a1 = a[0], b1 = b[0], cN = c[(long)(n - 1) * cs];
  if (b1 == 0.0) { rc = ORC_ESINGULAR; goto done; }
  for (int i = 0; i < n; ++i) {
    ap[i] = a[i * cs];
    bp[i] = b[i * cs];
    cp[i] = c[i * cs];
    rhs[i] = f[i * fs];
  }
  bp[0] = 2.0 * b1;
  bp[n - 1] = b[(long)(n - 1) * cs] + a1 * cN / b1;
  u[0] = -b1;
  u[n - 1] = cN;
  rc = thomas(n, ap, bp, cp, 1, rhs, y, chat);
  if (rc) goto done;
  rc = thomas(n, ap, bp, cp, 1, u, z, chat);
  if (rc) goto done;
  double vy = y[0] - (a1 / b1) * y[n - 1];
  double vz = z[0] - (a1 / b1) * z[n - 1];
  double den = 1.0 + vz;
  if (!(fabs(den) > 1e3 * 2.220446049250313e-16 * (1.0 + fabs(vz)))) { rc = ORC_ESINGULAR; goto done; }
  for (int i = 0; i < n; ++i) x[i * xs] = y[i] - (vy / den) * z[i];
done:
  free(bp); free(rhs); free(u); free(y); free(z); free(chat); free(ap); free(cp);
  return rc;
}

int oracle_tri_cyclic_batch(int n, int batch, int coef_mode, const double* a, const double* b,
                            const double* c, const double* f, double* x) {
  for (int s = 0; s < batch; ++s) {
    long off = coef_mode ? s : 0, cs = coef_mode ? batch : 1;
    int rc = oracle_tri_cyclic_solve(n, a + off, b + off, c + off, cs, f + s, batch, x + s, batch);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * General 2D stencil apply (Sec. 3.3): out(i,j) = sum over the box
 * dj in [-top, bottom], di in [-left, right] of w[(dj+top)*(left+right+1) +
 * (di+left)] * p(in(i+di, j+dj)), where p is the identity or, for the
 * function-pointer form used by the Cahn-Hilliard solver, p(c) = c^3 - c.
 * Fields are row-major with leading dimension ldx: v(i,j) = v[j*ldx + i].
 * periodic = 1 wraps indices in both directions; periodic = 0 computes only
 * points whose whole box lies inside the grid and leaves the others untouched.
 * ------------------------------------------------------------------------- */
int oracle_stencil_apply_2d(const double* in, double* out, int nx, int ny, int ldx,
                            const double* w, int left, int right, int top, int bottom,
                            int premap, int periodic) {
  if (nx <= 0 || ny <= 0 || ldx < nx || left < 0 || right < 0 || top < 0 || bottom < 0)
    return ORC_EINVAL;
  int bw = left + right + 1;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      if (!periodic && (i - left < 0 || i + right >= nx || j - top < 0 || j + bottom >= ny)) continue;
      double s = 0.0;
      for (int dj = -top; dj <= bottom; ++dj) {
        for (int di = -left; di <= right; ++di) {
          int ii = periodic ? wrap(i + di, nx) : i + di;
          int jj = periodic ? wrap(j + dj, ny) : j + dj;
          double v = in[(long)jj * ldx + ii];
          if (premap) v = v * v * v - v;
          s += w[(dj + top) * bw + (di + left)] * v;
        }
      }
      out[(long)j * ldx + i] = s;
    }
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * One ADI step of Eq. 3.1 (eq3:ch_adi) with D = 1, periodic on [0,lx)x[0,ly),
 * dx = lx/nx, dy = ly/ny (the periodic grid x_i = i dx of Sec. 4.2.1):
 *   Cbar = 2 C^n - C^{n-1}                 (reading: the BDF2 extrapolation)
 *   r = -(2/3)(C^n - C^{n-1}) - (2/3) gamma dt Lap_h^2 Cbar
 *       + (2/3) dt Lap_h (C^3 - C)^n        (reading: gamma restored on Lap^2)
 *   (I + (2/3) gamma dt dxxxx) w = r   row by row    (L_x)
 *   (I + (2/3) gamma dt dyyyy) v = w   column by column (L_y)
 *   C^{n+1} = Cbar + v.
 * Lap_h is the 5-point Laplacian, Lap_h^2 the 13-point biharmonic
 * dxxxx + 2 dxx dyy + dyyyy with the fourth difference (1,-4,6,-4,1)/dx^4 of
 * eq:1d_hyper_scheme and the cross stencil [1,-2,1;-2,4,-2;1,-2,1]/(dx^2 dy^2)
 * of fig3:stencil.  On return c_prev holds C^n and c_now C^{n+1}.
 * ------------------------------------------------------------------------- */
/* eta: NULL, or an nx*ny forcing field added to the PDE's right-hand side; in
 * the two-level scheme it enters r with the weight (2/3) dt of the explicit terms. */
static int ch_step_forced(int nx, int ny, double lx, double ly, double gamma, double dt,
                          double* c_now, double* c_prev, const double* eta) {
  if (nx < 5 || ny < 5 || !(lx > 0) || !(ly > 0) || !(dt > 0) || !(gamma >= 0)) return ORC_EINVAL;
  long np = (long)nx * ny;
  double dx = lx / nx, dy = ly / ny;
  double *cb = malloc(np * sizeof(double)), *r = malloc(np * sizeof(double));
  double *nl = malloc(np * sizeof(double)), *w = malloc(np * sizeof(double));
  double *ca = malloc(5 * (nx > ny ? nx : ny) * sizeof(double));
  int rc = ORC_OK;
  if (!cb || !r || !nl || !w || !ca) { rc = ORC_ENOMEM; goto done; }
  for (long p = 0; p < np; ++p) {
    cb[p] = 2.0 * c_now[p] - c_prev[p];
    nl[p] = c_now[p] * c_now[p] * c_now[p] - c_now[p];
  }
#define AT(v, i, j) (v)[(long)wrap((j), ny) * nx + wrap((i), nx)]
  double ix2 = 1.0 / (dx * dx), iy2 = 1.0 / (dy * dy);
  double ix4 = ix2 * ix2, iy4 = iy2 * iy2, ixy = ix2 * iy2;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double lapN = (AT(nl, i + 1, j) - 2.0 * AT(nl, i, j) + AT(nl, i - 1, j)) * ix2 +
                    (AT(nl, i, j + 1) - 2.0 * AT(nl, i, j) + AT(nl, i, j - 1)) * iy2;
      double dxxxx = (AT(cb, i - 2, j) - 4.0 * AT(cb, i - 1, j) + 6.0 * AT(cb, i, j) -
                      4.0 * AT(cb, i + 1, j) + AT(cb, i + 2, j)) * ix4;
      double dyyyy = (AT(cb, i, j - 2) - 4.0 * AT(cb, i, j - 1) + 6.0 * AT(cb, i, j) -
                      4.0 * AT(cb, i, j + 1) + AT(cb, i, j + 2)) * iy4;
      double dxxyy = (AT(cb, i - 1, j - 1) - 2.0 * AT(cb, i, j - 1) + AT(cb, i + 1, j - 1)
                      - 2.0 * AT(cb, i - 1, j) + 4.0 * AT(cb, i, j) - 2.0 * AT(cb, i + 1, j)
                      + AT(cb, i - 1, j + 1) - 2.0 * AT(cb, i, j + 1) + AT(cb, i + 1, j + 1)) * ixy;
      double bih = dxxxx + 2.0 * dxxyy + dyyyy;
      long p = (long)j * nx + i;
      r[p] = -(2.0 / 3.0) * (c_now[p] - c_prev[p]) - (2.0 / 3.0) * gamma * dt * bih +
             (2.0 / 3.0) * dt * lapN;
      if (eta) r[p] += (2.0 / 3.0) * dt * eta[p];
    }
  }
#undef AT
  /* L_x: rows are systems, unit stride inside a row. */
  double ax = (2.0 / 3.0) * gamma * dt * ix4;
  for (int i = 0; i < nx; ++i) {
    ca[i] = ax; ca[nx + i] = -4.0 * ax; ca[2 * nx + i] = 1.0 + 6.0 * ax;
    ca[3 * nx + i] = -4.0 * ax; ca[4 * nx + i] = ax;
  }
  for (int j = 0; j < ny; ++j) {
    rc = oracle_penta_cyclic_solve(nx, ca, ca + nx, ca + 2 * nx, ca + 3 * nx, ca + 4 * nx, 1,
                                   r + (long)j * nx, 1, w + (long)j * nx, 1);
    if (rc) goto done;
  }
  /* L_y: columns are systems, stride nx. */
  double ay = (2.0 / 3.0) * gamma * dt * iy4;
  for (int j = 0; j < ny; ++j) {
    ca[j] = ay; ca[ny + j] = -4.0 * ay; ca[2 * ny + j] = 1.0 + 6.0 * ay;
    ca[3 * ny + j] = -4.0 * ay; ca[4 * ny + j] = ay;
  }
  for (int i = 0; i < nx; ++i) {
    rc = oracle_penta_cyclic_solve(ny, ca, ca + ny, ca + 2 * ny, ca + 3 * ny, ca + 4 * ny, 1,
                                   w + i, nx, r + i, nx); /* v overwrites r */
    if (rc) goto done;
  }
  for (long p = 0; p < np; ++p) {
    double next = cb[p] + r[p];
    c_prev[p] = c_now[p];
    c_now[p] = next;
  }
done:
  free(cb); free(r); free(nl); free(w); free(ca);
  return rc;
}

int oracle_ch_step(int nx, int ny, double lx, double ly, double gamma, double dt,
                   double* c_now, double* c_prev) {
  return ch_step_forced(nx, ny, lx, ly, gamma, dt, c_now, c_prev, NULL);
}

int oracle_ch_run(int nx, int ny, double lx, double ly, double gamma, double dt, int nsteps,
                  double* c_now, double* c_prev) {
  for (int s = 0; s < nsteps; ++s) {
    int rc = oracle_ch_step(nx, ny, lx, ly, gamma, dt, c_now, c_prev);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Mass and discrete free energy (Sec. 2.4).  mass = sum c dx dy.
 * F_h = sum [ (1/4)(c^2 - 1)^2 + (gamma/2)(|D+x c|^2 + |D+y c|^2) ] dx dy with
 * forward differences and periodic wrap.  Reading: the printed bulk density
 * (1/2)(C^2-1)^2 does not have C^3 - C as its derivative, which the chemical
 * potential of eq2:ch and the decay law eq2:dFdt_ch require; (1/4)(C^2-1)^2 does.
 * ------------------------------------------------------------------------- */
int oracle_ch_diagnostics(int nx, int ny, double lx, double ly, double gamma, const double* c,
                          double* mass, double* energy) {
  if (nx < 1 || ny < 1) return ORC_EINVAL;
  double dx = lx / nx, dy = ly / ny, m = 0.0, e = 0.0;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double v = c[(long)j * nx + i];
      double gx = (c[(long)j * nx + wrap(i + 1, nx)] - v) / dx;
      double gy = (c[(long)wrap(j + 1, ny) * nx + i] - v) / dy;
      m += v;
      e += 0.25 * (v * v - 1.0) * (v * v - 1.0) + 0.5 * gamma * (gx * gx + gy * gy);
    }
  }
  *mass = m * dx * dy;
  *energy = e * dx * dy;
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Batched 1D Cahn-Hilliard step (Sec. 6.2.1, eq6:1Dnumerical): on [0, l) with
 * dx = l/n, for every system s of the interleaved batch c[i*batch + s],
 *   (I + sigma delta^4) C^{n+1} = C^n + alpha delta^2 (C^3 - C)^n,
 *   sigma = gamma dt / dx^4, alpha = dt / dx^2, periodic in i.
 * Reading: the printed right-hand side f_i omits C_i^n; eq6:1Dnumerical has it.
 * ------------------------------------------------------------------------- */
int oracle_ch1d_step(int n, int batch, double l, double gamma, double dt, double* c) {
  if (n < 5 || batch < 1 || !(l > 0) || !(dt > 0) || !(gamma >= 0)) return ORC_EINVAL;
  double dx = l / n, sigma = gamma * dt / (dx * dx * dx * dx), alpha = dt / (dx * dx);
  double *f = malloc(n * sizeof(double)), *x = malloc(n * sizeof(double)), *nl = malloc(n * sizeof(double));
  double *co = malloc(5 * n * sizeof(double));
  int rc = ORC_OK;
  if (!f || !x || !nl || !co) { rc = ORC_ENOMEM; goto done1; }
  for (int i = 0; i < n; ++i) {
    co[i] = sigma; co[n + i] = -4.0 * sigma; co[2 * n + i] = 1.0 + 6.0 * sigma;
    co[3 * n + i] = -4.0 * sigma; co[4 * n + i] = sigma;
  }
  for (int s = 0; s < batch; ++s) {
    for (int i = 0; i < n; ++i) {
      double v = c[(long)i * batch + s];
      nl[i] = v * v * v - v;
    }
    for (int i = 0; i < n; ++i)
      f[i] = c[(long)i * batch + s] + alpha * (nl[wrap(i - 1, n)] - 2.0 * nl[i] + nl[wrap(i + 1, n)]);
    rc = oracle_penta_cyclic_solve(n, co, co + n, co + 2 * n, co + 3 * n, co + 4 * n, 1, f, 1, x, 1);
    if (rc) goto done1;
    for (int i = 0; i < n; ++i) c[(long)i * batch + s] = x[i];
  }
done1:
  free(f); free(x); free(nl); free(co);
  return rc;
}

int oracle_ch1d_run(int n, int batch, double l, double gamma, double dt, int nsteps, double* c) {
  for (int k = 0; k < nsteps; ++k) {
    int rc = oracle_ch1d_step(n, batch, l, gamma, dt, c);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Crank-Nicolson benchmark steps on a batch of periodic 1D problems,
 * interleaved c[i*batch + s], dx = l/n:
 *  order 4, hyperdiffusion C_t = -kappa C_xxxx (Sec. 4.2.1, eq:1d_hyper_scheme):
 *    sigma = kappa dt / (2 dx^4),
 *    (sigma, -4 sigma, 1 + 6 sigma, -4 sigma, sigma) C^{n+1}
 *      = (-sigma, 4 sigma, 1 - 6 sigma, 4 sigma, -sigma) C^n;
 *  order 2, diffusion C_t = kappa C_xx (Sec. 5.3.2, eq5:1ddiffscheme):
 *    sigma = kappa dt / (2 dx^2),
 *    (-sigma, 1 + 2 sigma, -sigma) C^{n+1} = (sigma, 1 - 2 sigma, sigma) C^n.
 * ------------------------------------------------------------------------- */
int oracle_cn1d_run(int order, int n, int batch, double l, double kappa, double dt, int nsteps, double* c) {
  if ((order != 2 && order != 4) || n < (order == 4 ? 5 : 3) || batch < 1 || !(l > 0) || !(dt > 0) || !(kappa >= 0)) return ORC_EINVAL;
  double dx = l / n;
  double sigma = order == 4 ? kappa * dt / (2.0 * dx * dx * dx * dx) : kappa * dt / (2.0 * dx * dx);
  double *f = malloc(n * sizeof(double)), *x = malloc(n * sizeof(double)), *co = malloc(5 * n * sizeof(double));
  int rc = ORC_OK;
  if (!f || !x || !co) { rc = ORC_ENOMEM; goto done2; }
  for (int i = 0; i < n; ++i) {
    if (order == 4) {
      co[i] = sigma; co[n + i] = -4.0 * sigma; co[2 * n + i] = 1.0 + 6.0 * sigma;
      co[3 * n + i] = -4.0 * sigma; co[4 * n + i] = sigma;
    } else {
      co[i] = -sigma; co[n + i] = 1.0 + 2.0 * sigma; co[2 * n + i] = -sigma;
    }
  }
  for (int k = 0; k < nsteps; ++k) {
    for (int s = 0; s < batch; ++s) {
      for (int i = 0; i < n; ++i) {
#define CC(j) c[(long)wrap((j), n) * batch + s]
        if (order == 4)
          f[i] = -sigma * CC(i - 2) + 4.0 * sigma * CC(i - 1) + (1.0 - 6.0 * sigma) * CC(i) + 4.0 * sigma * CC(i + 1) -
                 sigma * CC(i + 2);
        else
          f[i] = sigma * CC(i - 1) + (1.0 - 2.0 * sigma) * CC(i) + sigma * CC(i + 1);
#undef CC
      }
      if (order == 4)
        rc = oracle_penta_cyclic_solve(n, co, co + n, co + 2 * n, co + 3 * n, co + 4 * n, 1, f, 1, x, 1);
      else
        rc = oracle_tri_cyclic_solve(n, co, co + n, co + 2 * n, 1, f, 1, x, 1);
      if (rc) goto done2;
      for (int i = 0; i < n; ++i) c[(long)i * batch + s] = x[i];
    }
  }
done2:
  free(f); free(x); free(co);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Cahn-Hilliard-Cook forcing (Sec. 7.7): C_t = D Lap(C^3 - C - gamma Lap C) + eta,
 * eta_ij = sqrt(sigma / (dx dy dt)) div_h rho_ij, rho a 2-vector field of N(0,1)
 * deviates drawn afresh every step by the Box-Muller transform of uniforms.
 * Readings: div_h is the backward difference
 *   (rho^x_ij - rho^x_{i-1,j}) / dx + (rho^y_ij - rho^y_{i,j-1}) / dy
 * (periodic), whose covariance is sigma/(dx dy dt) times minus the 5-point
 * Laplacian of a Kronecker delta, the discrete form of the stated correlation;
 * dx^2 of the prefactor is dx dy for unequal spacings.
 *
 * Uniforms come from the counter-based generator Philox4x64-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011):
 * 10 rounds, each (hi0, lo0) = M0 * x0, (hi1, lo1) = M1 * x2 (128-bit products),
 * x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0), with the key bumped by the
 * Weyl constants W0, W1 between rounds.
 * ------------------------------------------------------------------------- */
void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Normal deviates of step `step` for an nx*ny grid: rho[0 .. np-1] = rho^x,
 * rho[np .. 2np-1] = rho^y (row-major).  Points 2b and 2b+1 take the four words
 * of Philox(counter = (b, step, 0, 0), key = (seed, sim)); word w gives the
 * uniform u = (floor(w / 2^41) + 1/2) 2^-23 in (0, 1), and the pairs (u0, u1),
 * (u2, u3) give (rho^x, rho^y) of the two points by Box-Muller:
 *   rho^x = sqrt(-2 ln u_a) cos(2 pi u_b), rho^y = sqrt(-2 ln u_a) sin(2 pi u_b). */
int oracle_noise_normals(int nx, int ny, uint64_t seed, uint64_t sim, uint64_t step, double* rho) {
  if (nx < 1 || ny < 1) return ORC_EINVAL;
  long np = (long)nx * ny;
  const uint64_t key[2] = {seed, sim};
  for (long b = 0; 2 * b < np; ++b) {
    uint64_t ctr[4] = {(uint64_t)b, step, 0, 0}, w[4];
    oracle_philox4x64(ctr, key, w);
    for (int h = 0; h < 2; ++h) {
      long p = 2 * b + h;
      if (p >= np) break;
      double ua = ((double)(w[2 * h] >> 41) + 0.5) * 0x1p-23;
      double ub = ((double)(w[2 * h + 1] >> 41) + 0.5) * 0x1p-23;
      double rad = sqrt(-2.0 * log(ua));
      rho[p] = rad * cos(6.283185307179586 * ub); /* 2 pi */
      rho[np + p] = rad * sin(6.283185307179586 * ub);
    }
  }
  return ORC_OK;
}

/* eta = sqrt(sigma / (dx dy dt)) div_h rho (reading above). */
int oracle_cook_forcing(int nx, int ny, double lx, double ly, double dt, double sigma, const double* rho,
                        double* eta) {
  if (nx < 2 || ny < 2 || !(lx > 0) || !(ly > 0) || !(dt > 0) || !(sigma >= 0)) return ORC_EINVAL;
  long np = (long)nx * ny;
  double dx = lx / nx, dy = ly / ny, amp = sqrt(sigma / (dx * dy * dt));
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      long p = (long)j * nx + i;
      double div = (rho[p] - rho[(long)j * nx + wrap(i - 1, nx)]) / dx +
                   (rho[np + p] - rho[np + (long)wrap(j - 1, ny) * nx + i]) / dy;
      eta[p] = amp * div;
    }
  return ORC_OK;
}

/* One Cahn-Hilliard-Cook step with the given deviates rho (2 nx ny values). */
int oracle_ch_cook_step(int nx, int ny, double lx, double ly, double gamma, double dt, double sigma,
                        const double* rho, double* c_now, double* c_prev) {
  double* eta = malloc((size_t)nx * ny * sizeof(double));
  if (!eta) return ORC_ENOMEM;
  int rc = oracle_cook_forcing(nx, ny, lx, ly, dt, sigma, rho, eta);
  if (!rc) rc = ch_step_forced(nx, ny, lx, ly, gamma, dt, c_now, c_prev, eta);
  free(eta);
  return rc;
}

/* nsteps steps, the deviates of step k (k = step0 ..) drawn by oracle_noise_normals. */
int oracle_ch_cook_run(int nx, int ny, double lx, double ly, double gamma, double dt, double sigma, uint64_t seed,
                       uint64_t sim, uint64_t step0, int nsteps, double* c_now, double* c_prev) {
  double* rho = malloc(2 * (size_t)nx * ny * sizeof(double));
  if (!rho) return ORC_ENOMEM;
  int rc = ORC_OK;
  for (int k = 0; k < nsteps && !rc; ++k) {
    rc = oracle_noise_normals(nx, ny, seed, sim, step0 + (uint64_t)k, rho);
    if (!rc) rc = oracle_ch_cook_step(nx, ny, lx, ly, gamma, dt, sigma, rho, c_now, c_prev);
  }
  free(rho);
  return rc;
}
