/*
 * mgfr_oracle.c -- plain, slow FP64 CPU reference ("oracle") for the f(R)
 * field solver of Puchwein, Baldi & Springel, "Modified-Gravity-GADGET"
 * (arXiv:1305.2418).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is never part of the product path:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only through the seeded input generator.
 *
 * Everything is FP64, round-to-nearest, compiled without contraction
 * (-ffp-contract=off) and without fast-math, written for legibility: loops
 * over cells in the order the paper describes, no blocking, no fusion.
 * Loops whose iterations write distinct cells and read only values no other
 * iteration of the same loop writes (one colour of a red-black sweep, a
 * residual, a restriction or prolongation) may run on several threads
 * (OpenMP, orc_set_threads); sums and the particle deposit stay sequential,
 * so every result is bit-identical to the single-threaded run.
 *
 * What it computes (paper section / equation in brackets):
 *   - model constants: background curvature R(a) and background field
 *     fR(a) of the Hu-Sawicki model [Sec. 2, Eqs. (10), (11)];
 *   - the discrete operator L and source f of the field equation for
 *     u = ln(fR / fR_bar) [Sec. 3.2, Eqs. (15), (16), (22)], in comoving
 *     units (see model_make below);
 *   - Newton-Gauss-Seidel point updates in red-black order
 *     [Sec. 3.3, Eq. (23)];
 *   - FAS multigrid V-cycles down to a 4^3 grid [Sec. 3.3, Eqs.
 *     (27), (29), steps 1-8];
 *   - the refinement hierarchy from particle counts, adaptive cloud-in-cell
 *     mass assignment and upward mass sums [Sec. 3.1];
 *   - one-way solves of refined levels with fixed ghost cells prolonged from
 *     the parent level [Sec. 3.3, steps 9-12];
 *   - f_R = fR_bar e^u and the extra force (c^2/2) grad f_R [Sec. 2,
 *     Eq. (13)], on cells and interpolated back to particles;
 *   - the effective mass density delta rho_eff [Sec. 2.4, Eq.
 *     (31)] per cell, and its share on a nested PM grid by
 *     overlapping volume [Sec. 2.4].
 *
 * Readings where the paper is silent:
 *   - dL/du is the full derivative of the discrete L_i w.r.t. u_i with the
 *     neighbours fixed; the Newton step is clamped to |du| <= step_cap (the
 *     clamp changes the path, never the fixed point);
 *   - the residual is restricted with the same 8-child average as u;
 *   - the stopping test is ||f - L(u)||_2 <= tol * ||f||_2 (zero-start
 *     residual, since L(0) = 0); when f == 0 the initial residual is used;
 *   - general n: nonlinearity 1 - exp(-u/(n+1)), fR_bar ~ R^-(n+1);
 *   - refinement: a cell at level l < lmax is flagged when its particle count
 *     exceeds refine_count, flags are dilated by one cell over the 26
 *     neighbours, and every flagged cell gets all 8 children [Sec. 3.1];
 *   - a ghost takes the linear reconstruction of its parent's value, with a
 *     gradient component set to 0 where one of the parent's two neighbours
 *     on that axis does not exist;
 *   - refined levels are relaxed by plain red-black NGS until the stopping
 *     test holds (the paper's masked multigrid only accelerates this);
 *   - force: central differences of f_R per level (ghosts at patch edges),
 *     a_MG / c^2 = grad_x f_R / (2a) with x comoving in Mpc/h, and particle
 *     values gathered with the same overlap weights as the mass assignment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the parallel loops (<= 0: all available); returns the count
 * in use.  Without OpenMP the oracle runs on one thread. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n <= 0) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}

#define ORC_MAXLEV 16
#define ORC_CLIGHT_OVER_H0 2997.92458 /* c / H0 in Mpc/h */

/* ------------------------------------------------------------------------ */
/* Model constants [Sec. 2].                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  double omega_m, omega_l, a;
  double Rt;    /* R_bar(a) / (3 H0^2) = Om a^-3 + 4 OL                       */
  double fbar;  /* fR_bar(a) < 0                                             */
  double alpha; /* a^2 (H0/c)^2 / fR_bar(a)  [(h/Mpc)^2], negative           */
  double src;   /* f = src * delta with src = -alpha Om a^-3                 */
  double fr0_abs;
  int n;
} orc_model;

/*
 * Dividing the physical field equation [Eq. (16)] by a^-2 (the
 * physical Laplacian is a^-2 times the comoving one) and using
 * R_bar = 3 H0^2 Rt [Sec. 2] and 8 pi G rho_bar = 3 H0^2 Om a^-3 gives
 *     lap_x e^u + alpha [Rt (1 - e^{-u/(n+1)}) + Om a^-3 delta] = 0,
 * with alpha = a^2 (H0/c)^2 / fR_bar(a).  fR_bar(a) = -|fR0| (Rt(1)/Rt(a))^{n+1}
 * [Eq. (10) for n = 1; the exponent n+1 follows from Eq.
 * (7)].  Flatness: OL = 1 - Om.
 */
static orc_model model_make(double omega_m, double fr0_abs, int n, double a) {
  orc_model m;
  double kappa = 1.0 / (ORC_CLIGHT_OVER_H0 * ORC_CLIGHT_OVER_H0);
  m.omega_m = omega_m;
  m.fr0_abs = fr0_abs;
  m.omega_l = 1.0 - omega_m;
  m.a = a;
  m.n = n;
  m.Rt = omega_m / (a * a * a) + 4.0 * m.omega_l;
  double Rt1 = omega_m + 4.0 * m.omega_l;
  m.fbar = -fr0_abs * pow(Rt1 / m.Rt, (double)(n + 1));
  m.alpha = a * a * kappa / m.fbar;
  m.src = -m.alpha * omega_m / (a * a * a);
  return m;
}

void orc_model_constants(double omega_m, double fr0_abs, int n, double a, double* out4) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  out4[0] = m.Rt;
  out4[1] = m.fbar;
  out4[2] = m.alpha;
  out4[3] = m.src;
}

/*
 * Effective mass density [Sec. 2.4, Eqs. (30) and (31)]:
 * delta rho_eff = delta rho / 3 - delta R / (24 pi G),
 * with delta R = R_bar ((fR_bar / f_R)^{1/(n+1)} - 1) [Eq. (11), general n
 * by Eq. (7)] = R_bar (e^{-u/(n+1)} - 1).  In units of the mean
 * matter density, with R_bar = 3 H0^2 Rt and 24 pi G rho_bar = 9 H0^2 Om a^-3:
 *     delta_eff = delta / 3 + Rt / (3 Om a^-3) (1 - e^{-u/(n+1)}).
 * Per cell of any level (u, delta, out: n values).
 */
void orc_effective_density(long long ncell, const double* u, const double* delta,
                           double omega_m, double fr0_abs, int n, double a, double* out) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  const double rho = omega_m / (a * a * a);
  for (long long c = 0; c < ncell; ++c)
    out[c] = delta[c] / 3.0 + m.Rt / (3.0 * rho) * (1.0 - exp(-u[c] / (m.n + 1)));
}

/* ------------------------------------------------------------------------ */
/* Dense periodic grids (the levels that cover the whole box).              */
/* Layout: C order a[i][j][k], i along x (slowest), k along z (fastest).    */
/* ------------------------------------------------------------------------ */

static long didx(int N, int i, int j, int k) {
  i = (i % N + N) % N;
  j = (j % N + N) % N;
  k = (k % N + N) % N;
  return ((long)i * N + j) * N + k;
}

/*
 * L_ijk [Sec. 3.2]: (1/h^2) sum over the three axes of
 *   b_- u_- + b_+ u_+ - (b_- + b_+) u_c,  b_{+-} = (e^{u_{+-}} + e^{u_c}) / 2,
 * plus alpha Rt (1 - e^{-u_c/(n+1)}).
 */
static double dense_L(const double* u, int N, int i, int j, int k, double ih2,
                      const orc_model* m) {
  double uc = u[didx(N, i, j, k)];
  double Ec = exp(uc);
  const int di[3] = {1, 0, 0}, dj[3] = {0, 1, 0}, dk[3] = {0, 0, 1};
  double lap = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double um = u[didx(N, i - di[ax], j - dj[ax], k - dk[ax])];
    double up = u[didx(N, i + di[ax], j + dj[ax], k + dk[ax])];
    double bm = 0.5 * (exp(um) + Ec);
    double bp = 0.5 * (exp(up) + Ec);
    lap += bm * um + bp * up - (bm + bp) * uc;
  }
  return lap * ih2 + m->alpha * m->Rt * (1.0 - exp(-uc / (m->n + 1)));
}

/*
 * d L_ijk / d u_ijk with the six neighbours held fixed (the paper does not
 * print it).  For one neighbour j: d/du_c [b (u_j - u_c)] =
 * (e^{u_c}/2)(u_j - u_c) - b.  Nonlinear part: alpha Rt/(n+1) e^{-u_c/(n+1)}.
 */
static double dense_dL(const double* u, int N, int i, int j, int k, double ih2,
                       const orc_model* m) {
  double uc = u[didx(N, i, j, k)];
  double Ec = exp(uc);
  const int di[3] = {1, 0, 0}, dj[3] = {0, 1, 0}, dk[3] = {0, 0, 1};
  double d = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    for (int s = -1; s <= 1; s += 2) {
      double un = u[didx(N, i + s * di[ax], j + s * dj[ax], k + s * dk[ax])];
      double b = 0.5 * (exp(un) + Ec);
      d += 0.5 * Ec * (un - uc) - b;
    }
  }
  return d * ih2 + m->alpha * m->Rt / (m->n + 1) * exp(-uc / (m->n + 1));
}

/* Newton-Gauss-Seidel red-black sweep [Eq. (23)]: red cells
 * ((i+j+k) even) first, then black. */
static void dense_rb_sweep(double* u, const double* f, int N, double h, const orc_model* m,
                           double step_cap) {
  double ih2 = 1.0 / (h * h);
  for (int colour = 0; colour < 2; ++colour)
#pragma omp parallel for schedule(static) if (N >= 32)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
          if (((i + j + k) & 1) != colour) continue;
          long c = didx(N, i, j, k);
          double step = (dense_L(u, N, i, j, k, ih2, m) - f[c]) / dense_dL(u, N, i, j, k, ih2, m);
          if (step > step_cap) step = step_cap;
          if (step < -step_cap) step = -step_cap;
          u[c] -= step;
        }
}

static void dense_residual(const double* u, const double* f, int N, double h, const orc_model* m,
                           double* r) {
  double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static) if (N >= 32)
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        long c = didx(N, i, j, k);
        r[c] = f[c] - dense_L(u, N, i, j, k, ih2, m);
      }
}

static double norm2(const double* a, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * a[i];
  return sqrt(s);
}

static double normmax(const double* a, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i)
    if (fabs(a[i]) > s) s = fabs(a[i]);
  return s;
}

/* Restriction R [Sec. 3.3]: parent value = average of its 8 daughters. */
static void dense_restrict(const double* fine, int Nf, double* coarse) {
  int Nc = Nf / 2;
#pragma omp parallel for schedule(static) if (Nc >= 32)
  for (int I = 0; I < Nc; ++I)
    for (int J = 0; J < Nc; ++J)
      for (int K = 0; K < Nc; ++K) {
        double s = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) s += fine[didx(Nf, 2 * I + a, 2 * J + b, 2 * K + c)];
        coarse[didx(Nc, I, J, K)] = s / 8.0;
      }
}

/*
 * Prolongation P [Sec. 3.3], added onto the fine field: straight injection,
 * or linear reconstruction from the parent's central-difference gradient.
 * A daughter sits a quarter of the parent's width from its centre, so
 *   child = parent + sum_d s_d (c_{+d} - c_{-d}) / 8,   s_d = +-1.
 */
static void dense_prolong_add(const double* coarse, int Nc, double* fine, int linear) {
  int Nf = 2 * Nc;
#pragma omp parallel for schedule(static) if (Nf >= 32)
  for (int i = 0; i < Nf; ++i)
    for (int j = 0; j < Nf; ++j)
      for (int k = 0; k < Nf; ++k) {
        int I = i / 2, J = j / 2, K = k / 2;
        double v = coarse[didx(Nc, I, J, K)];
        if (linear) {
          double sx = (i & 1) ? 1.0 : -1.0, sy = (j & 1) ? 1.0 : -1.0, sz = (k & 1) ? 1.0 : -1.0;
          v += sx * (coarse[didx(Nc, I + 1, J, K)] - coarse[didx(Nc, I - 1, J, K)]) / 8.0;
          v += sy * (coarse[didx(Nc, I, J + 1, K)] - coarse[didx(Nc, I, J - 1, K)]) / 8.0;
          v += sz * (coarse[didx(Nc, I, J, K + 1)] - coarse[didx(Nc, I, J, K - 1)]) / 8.0;
        }
        fine[didx(Nf, i, j, k)] += v;
      }
}

typedef struct {
  int n_pre, n_post, prolong_linear, coarse_max_sweeps;
  double step_cap, coarse_rel;
  long long updates; /* cell updates performed, all levels */
} orc_mg;

/* Direct NGS on the 4^3 grid [Sec. 3.3, step 5]: sweeps until the max
 * residual has dropped by coarse_rel, at most coarse_max_sweeps. */
static void dense_coarse_solve(double* u, const double* f, int N, double h, const orc_model* m,
                               orc_mg* mg) {
  long n = (long)N * N * N;
  double* r = (double*)malloc(sizeof(double) * n);
  dense_residual(u, f, N, h, m, r);
  double r0 = normmax(r, n);
  for (int s = 0; s < mg->coarse_max_sweeps && r0 > 0.0; ++s) {
    dense_rb_sweep(u, f, N, h, m, mg->step_cap);
    mg->updates += n;
    dense_residual(u, f, N, h, m, r);
    if (normmax(r, n) <= mg->coarse_rel * r0) break;
  }
  free(r);
}

/*
 * One FAS V-cycle on the dense level of size N [Sec. 3.3, steps 3-7]:
 * pre-smooth; restrict u and the residual; coarse RHS
 * f^{2h} = L^{2h}(R u) + R(f - L(u)) [Eq. (27)]; solve the coarse
 * problem (recursively while the coarse grid is larger than 4^3, directly on
 * 4^3); correct u += P(u^{2h} - R u) [Eq. (29)]; post-smooth.
 */
static void dense_vcycle(double* u, const double* f, int N, double h, const orc_model* m,
                         orc_mg* mg) {
  long n = (long)N * N * N;
  for (int s = 0; s < mg->n_pre; ++s) {
    dense_rb_sweep(u, f, N, h, m, mg->step_cap);
    mg->updates += n;
  }
  int Nc = N / 2;
  long nc = (long)Nc * Nc * Nc;
  double hc = 2.0 * h;
  double* r = (double*)malloc(sizeof(double) * n);
  double* uc = (double*)malloc(sizeof(double) * nc);
  double* uc0 = (double*)malloc(sizeof(double) * nc);
  double* rc = (double*)malloc(sizeof(double) * nc);
  double* fc = (double*)malloc(sizeof(double) * nc);
  dense_residual(u, f, N, h, m, r);
  dense_restrict(u, N, uc);
  dense_restrict(r, N, rc);
  double ihc2 = 1.0 / (hc * hc);
#pragma omp parallel for schedule(static) if (Nc >= 32)
  for (int I = 0; I < Nc; ++I)
    for (int J = 0; J < Nc; ++J)
      for (int K = 0; K < Nc; ++K) {
        long c = didx(Nc, I, J, K);
        fc[c] = dense_L(uc, Nc, I, J, K, ihc2, m) + rc[c];
      }
  memcpy(uc0, uc, sizeof(double) * nc);
  if (Nc > 4)
    dense_vcycle(uc, fc, Nc, hc, m, mg);
  else
    dense_coarse_solve(uc, fc, Nc, hc, m, mg);
  for (long c = 0; c < nc; ++c) uc[c] -= uc0[c];
  dense_prolong_add(uc, Nc, u, mg->prolong_linear);
  for (int s = 0; s < mg->n_post; ++s) {
    dense_rb_sweep(u, f, N, h, m, mg->step_cap);
    mg->updates += n;
  }
  free(r);
  free(uc);
  free(uc0);
  free(rc);
  free(fc);
}

/* f_ijk [Sec. 3.2] in comoving units: f = -alpha Om a^-3 delta. */
static void make_source(const double* delta, long n, const orc_model* m, double* f) {
  for (long c = 0; c < n; ++c) f[c] = m->src * delta[c];
}

/*
 * Solve L(u) = f on a periodic N^3 grid by FAS V-cycles [Sec. 3.3 steps 1-8].
 * u holds the initial guess on entry and the solution on exit.
 * stats (nullable, 8 doubles): [0] V-cycles, [1] ||r0||_2, [2] ||r||_2,
 * [3] max|r|, [4] ||f||_2, [5] cell updates, [6] converged flag.
 * Returns 0 when the stopping test held, 1 otherwise.
 */
int orc_solve_dense_f(int N, double box, const double* f, double omega_m, double fr0_abs, int n,
                      double a, double* u, double tol, int max_vcycles, int n_pre, int n_post,
                      int prolong_linear, double step_cap, double* stats) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  long nc = (long)N * N * N;
  double h = box / N;
  orc_mg mg = {n_pre, n_post, prolong_linear, 200, step_cap, 1e-12, 0};
  double* r = (double*)malloc(sizeof(double) * nc);
  double fn = norm2(f, nc);
  dense_residual(u, f, N, h, &m, r);
  double r0 = norm2(r, nc);
  double target = tol * (fn > 0.0 ? fn : r0);
  double rn = r0;
  int it = 0;
  while (rn > target && it < max_vcycles) {
    dense_vcycle(u, f, N, h, &m, &mg);
    ++it;
    dense_residual(u, f, N, h, &m, r);
    rn = norm2(r, nc);
  }
  if (stats) {
    stats[0] = it;
    stats[1] = r0;
    stats[2] = rn;
    stats[3] = normmax(r, nc);
    stats[4] = fn;
    stats[5] = (double)mg.updates;
    stats[6] = rn <= target ? 1.0 : 0.0;
  }
  free(r);
  return rn <= target ? 0 : 1;
}

int orc_solve_dense(int N, double box, const double* delta, double omega_m, double fr0_abs,
                    int n, double a, double* u, double tol, int max_vcycles, int n_pre, int n_post,
                    int prolong_linear, double step_cap, double* stats) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  long nc = (long)N * N * N;
  double* f = (double*)malloc(sizeof(double) * nc);
  make_source(delta, nc, &m, f);
  int rc = orc_solve_dense_f(N, box, f, omega_m, fr0_abs, n, a, u, tol, max_vcycles, n_pre,
                             n_post, prolong_linear, step_cap, stats);
  free(f);
  return rc;
}

/* r = f - L(u) on a dense periodic grid, with f = src * delta. */
void orc_residual_dense(int N, double box, const double* delta, double omega_m, double fr0_abs,
                        int n, double a, const double* u, double* r) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  long nc = (long)N * N * N;
  double* f = (double*)malloc(sizeof(double) * nc);
  make_source(delta, nc, &m, f);
  dense_residual(u, f, N, box / N, &m, r);
  free(f);
}

/* L(u) alone on a dense periodic grid (used to manufacture right-hand sides). */
void orc_apply_L_dense(int N, double box, double omega_m, double fr0_abs, int n, double a,
                       const double* u, double* out) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  double h = box / N, ih2 = 1.0 / (h * h);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) out[didx(N, i, j, k)] = dense_L(u, N, i, j, k, ih2, &m);
}

/* L(u) and r = f - L(u) at selected cells only (for spot checks at sizes the
 * full oracle solve does not reach). */
void orc_residual_dense_at(int N, double box, double omega_m, double fr0_abs, int n, double a,
                           const double* u, const double* delta, const long long* cells,
                           long long ncells, double* r) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  double h = box / N, ih2 = 1.0 / (h * h);
  for (long long q = 0; q < ncells; ++q) {
    long long c = cells[q];
    int k = (int)(c % N), j = (int)((c / N) % N), i = (int)(c / ((long long)N * N));
    r[q] = m.src * delta[c] - dense_L(u, N, i, j, k, ih2, &m);
  }
}

/*
 * Field and force on a dense periodic level [Sec. 2, Eq. (13)]:
 * fR = fR_bar e^u; a_MG / c^2 = grad_x fR / (2a), the gradient by central
 * differences.  acc layout: [3][N^3] (component-major).
 */
void orc_force_dense(int N, double box, double omega_m, double fr0_abs, int n, double a,
                     const double* u, double* fr, double* acc) {
  orc_model m = model_make(omega_m, fr0_abs, n, a);
  long nc = (long)N * N * N;
  double h = box / N;
  for (long c = 0; c < nc; ++c) fr[c] = m.fbar * exp(u[c]);
  if (!acc) return;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        long c = didx(N, i, j, k);
        double gx = (fr[didx(N, i + 1, j, k)] - fr[didx(N, i - 1, j, k)]) / (2.0 * h);
        double gy = (fr[didx(N, i, j + 1, k)] - fr[didx(N, i, j - 1, k)]) / (2.0 * h);
        double gz = (fr[didx(N, i, j, k + 1)] - fr[didx(N, i, j, k - 1)]) / (2.0 * h);
        acc[0 * nc + c] = gx / (2.0 * a);
        acc[1 * nc + c] = gy / (2.0 * a);
        acc[2 * nc + c] = gz / (2.0 * a);
      }
}

/* ------------------------------------------------------------------------ */
/* Adaptive hierarchy [Sec. 3.1] and refined-level solves [Sec. 3.3].       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int N0, nlev, lmax, refine_count;
  double box;
  long long Np;
  double* t; /* particle positions in base-cell units, wrapped to [0, N0) */
  /* per level */
  long long ncell[ORC_MAXLEV];
  long long noct[ORC_MAXLEV];   /* level >= 1 */
  int64_t* keys[ORC_MAXLEV];    /* level >= 1: sorted parent linear indices */
  int* count[ORC_MAXLEV];       /* particles per cell (nearest-grid-point) */
  unsigned char* refined[ORC_MAXLEV];
  double* mass[ORC_MAXLEV];     /* in units of the particle mass */
  double* u[ORC_MAXLEV];
  double* f[ORC_MAXLEV];
  int f_custom[ORC_MAXLEV];
  orc_model model;
  int have_model;
} orc_amr;

static int64_t lev_dim(const orc_amr* A, int l) { return (int64_t)A->N0 << l; }

static int64_t wrapi(int64_t i, int64_t N) { return ((i % N) + N) % N; }

/*
 * Position of a particle in base-cell units, wrapped periodically into
 * [0, N0).  The cell index at level l is floor(t * 2^l); scaling by a power of
 * two is exact, so the levels nest exactly.
 */
static double wrap_coord(double x, double inv, double N0) {
  double t = x * inv;
  if (t < 0.0 || t >= N0) {
    t = t - N0 * floor(t / N0);
    if (t >= N0 || t < 0.0) t = 0.0;
  }
  return t;
}

static long long find_oct(const orc_amr* A, int l, int64_t key) {
  long long lo = 0, hi = A->noct[l] - 1;
  const int64_t* k = A->keys[l];
  while (lo <= hi) {
    long long mid = (lo + hi) / 2;
    if (k[mid] == key) return mid;
    if (k[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Cell index of level-l cell (I,J,K) (periodically wrapped), or -1 if the
 * cell does not exist at level l. Within an oct: child = 4 di + 2 dj + dk. */
static long long find_cell(const orc_amr* A, int l, int64_t I, int64_t J, int64_t K) {
  if (l >= A->nlev) return -1;
  int64_t N = lev_dim(A, l);
  I = wrapi(I, N);
  J = wrapi(J, N);
  K = wrapi(K, N);
  if (l == 0) return (I * N + J) * N + K;
  int64_t Np = N / 2;
  int64_t key = ((I >> 1) * Np + (J >> 1)) * Np + (K >> 1);
  long long o = find_oct(A, l, key);
  if (o < 0) return -1;
  return o * 8 + ((I & 1) << 2) + ((J & 1) << 1) + (K & 1);
}

static void cell_coords(const orc_amr* A, int l, long long c, int64_t* I, int64_t* J, int64_t* K) {
  int64_t N = lev_dim(A, l);
  if (l == 0) {
    *K = c % N;
    *J = (c / N) % N;
    *I = c / (N * N);
    return;
  }
  int64_t Np = N / 2;
  int64_t key = A->keys[l][c / 8];
  int ch = (int)(c % 8);
  int64_t pk = key % Np, pj = (key / Np) % Np, pi = key / (Np * Np);
  *I = 2 * pi + ((ch >> 2) & 1);
  *J = 2 * pj + ((ch >> 1) & 1);
  *K = 2 * pk + (ch & 1);
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

static void count_level(orc_amr* A, int l) {
  long long n = A->ncell[l];
  A->count[l] = (int*)calloc((size_t)n, sizeof(int));
  for (long long p = 0; p < A->Np; ++p) {
    const double* t = A->t + 3 * p;
    int64_t I = (int64_t)floor(ldexp(t[0], l));
    int64_t J = (int64_t)floor(ldexp(t[1], l));
    int64_t K = (int64_t)floor(ldexp(t[2], l));
    long long c = find_cell(A, l, I, J, K);
    if (c >= 0) A->count[l][c] += 1;
  }
}

/*
 * Build the refinement hierarchy [Sec. 3.1].  A level-l cell with l < lmax is
 * flagged when it holds more than refine_count particles; flags are dilated
 * over the 26 neighbours that exist at level l; each flagged cell is refined
 * into a full oct of 8 daughters ("create all 8 siblings").
 */
void* orc_amr_create(const double* pos, long long Np, int N0, double box, int lmax,
                     int refine_count) {
  orc_amr* A = (orc_amr*)calloc(1, sizeof(orc_amr));
  A->N0 = N0;
  A->box = box;
  A->Np = Np;
  A->lmax = lmax;
  A->refine_count = refine_count;
  A->t = (double*)malloc(sizeof(double) * 3 * (size_t)(Np > 0 ? Np : 1));
  double inv = (double)N0 / box;
  for (long long p = 0; p < 3 * Np; ++p) A->t[p] = wrap_coord(pos[p], inv, (double)N0);
  A->nlev = 1;
  A->ncell[0] = (long long)N0 * N0 * N0;
  count_level(A, 0);
  for (int l = 0; l < lmax && l + 1 < ORC_MAXLEV; ++l) {
    long long n = A->ncell[l];
    A->refined[l] = (unsigned char*)calloc((size_t)n, 1);
    for (long long c = 0; c < n; ++c) {
      if (A->count[l][c] <= refine_count) continue;
      int64_t I, J, K;
      cell_coords(A, l, c, &I, &J, &K);
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int d = -1; d <= 1; ++d) {
            long long nb = find_cell(A, l, I + a, J + b, K + d);
            if (nb >= 0) A->refined[l][nb] = 1;
          }
    }
    long long nref = 0;
    for (long long c = 0; c < n; ++c) nref += A->refined[l][c];
    if (nref == 0) break;
    int64_t N = lev_dim(A, l);
    int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * (size_t)nref);
    long long q = 0;
    for (long long c = 0; c < n; ++c) {
      if (!A->refined[l][c]) continue;
      int64_t I, J, K;
      cell_coords(A, l, c, &I, &J, &K);
      keys[q++] = (I * N + J) * N + K;
    }
    qsort(keys, (size_t)nref, sizeof(int64_t), cmp_i64);
    A->keys[l + 1] = keys;
    A->noct[l + 1] = nref;
    A->ncell[l + 1] = 8 * nref;
    A->nlev = l + 2;
    count_level(A, l + 1);
  }
  for (int l = 0; l < A->nlev; ++l) {
    if (!A->refined[l]) A->refined[l] = (unsigned char*)calloc((size_t)A->ncell[l], 1);
    A->mass[l] = (double*)calloc((size_t)A->ncell[l], sizeof(double));
    A->u[l] = (double*)calloc((size_t)A->ncell[l], sizeof(double));
    A->f[l] = (double*)calloc((size_t)A->ncell[l], sizeof(double));
  }
  return A;
}

void orc_amr_free(void* h) {
  orc_amr* A = (orc_amr*)h;
  if (!A) return;
  for (int l = 0; l < ORC_MAXLEV; ++l) {
    free(A->keys[l]);
    free(A->count[l]);
    free(A->refined[l]);
    free(A->mass[l]);
    free(A->u[l]);
    free(A->f[l]);
  }
  free(A->t);
  free(A);
}

int orc_amr_nlev(void* h) { return ((orc_amr*)h)->nlev; }
long long orc_amr_ncell(void* h, int l) { return ((orc_amr*)h)->ncell[l]; }
long long orc_amr_noct(void* h, int l) { return l == 0 ? 0 : ((orc_amr*)h)->noct[l]; }

void orc_amr_keys(void* h, int l, long long* out) {
  orc_amr* A = (orc_amr*)h;
  for (long long o = 0; o < A->noct[l]; ++o) out[o] = A->keys[l][o];
}
void orc_amr_counts(void* h, int l, int* out) {
  orc_amr* A = (orc_amr*)h;
  memcpy(out, A->count[l], sizeof(int) * (size_t)A->ncell[l]);
}
void orc_amr_refined(void* h, int l, unsigned char* out) {
  orc_amr* A = (orc_amr*)h;
  memcpy(out, A->refined[l], (size_t)A->ncell[l]);
}

/* Level of the deepest existing cell that contains base-unit position t. */
static int leaf_level(const orc_amr* A, const double* t) {
  int l = 0;
  for (;;) {
    long long c = find_cell(A, l, (int64_t)floor(ldexp(t[0], l)), (int64_t)floor(ldexp(t[1], l)),
                            (int64_t)floor(ldexp(t[2], l)));
    if (!A->refined[l][c]) return l;
    ++l;
  }
}

/*
 * Visit the leaf cells that a box [lo,hi] (base-cell units, not wrapped)
 * lying inside level-l position (I,J,K) overlaps, calling back with the
 * overlap volume in base-cell units.  If the position exists and is refined
 * the box is split among the 8 daughters; if it does not exist the whole box
 * goes to the deepest existing ancestor, which is a leaf.
 */
typedef void (*leaf_cb)(orc_amr* A, int l, long long c, double vol, void* ctx);

static void visit_region(orc_amr* A, int l, int64_t I, int64_t J, int64_t K, const double lo[3],
                         const double hi[3], leaf_cb cb, void* ctx) {
  double vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  if (!(vol > 0.0)) return;
  long long c = find_cell(A, l, I, J, K);
  if (c < 0) {
    int lu = l;
    int64_t Iu = I, Ju = J, Ku = K;
    while (c < 0) {
      --lu;
      Iu = (int64_t)floor(Iu / 2.0);
      Ju = (int64_t)floor(Ju / 2.0);
      Ku = (int64_t)floor(Ku / 2.0);
      c = find_cell(A, lu, Iu, Ju, Ku);
    }
    cb(A, lu, c, vol, ctx);
    return;
  }
  if (!A->refined[l][c]) {
    cb(A, l, c, vol, ctx);
    return;
  }
  double w = ldexp(1.0, -(l + 1)); /* daughter width, base units */
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 2; ++d) {
        int64_t ci = 2 * I + a, cj = 2 * J + b, ck = 2 * K + d;
        double clo[3] = {ci * w, cj * w, ck * w};
        double nlo[3], nhi[3];
        int empty = 0;
        for (int ax = 0; ax < 3; ++ax) {
          nlo[ax] = lo[ax] > clo[ax] ? lo[ax] : clo[ax];
          nhi[ax] = hi[ax] < clo[ax] + w ? hi[ax] : clo[ax] + w;
          if (!(nhi[ax] > nlo[ax])) empty = 1;
        }
        if (!empty) visit_region(A, l + 1, ci, cj, ck, nlo, nhi, cb, ctx);
      }
}

/*
 * Adaptive cloud-in-cell [Sec. 3.1]: the particle is a cube whose side is
 * that of the AMR cell it resides in (its leaf cell); every leaf cell gets the
 * overlapping fraction of the particle mass.  The cube is cut at the level-l
 * grid into (up to) 8 pieces, each then handed to visit_region.
 */
static void visit_particle(orc_amr* A, const double* t, leaf_cb cb, void* ctx) {
  int l = leaf_level(A, t);
  double s = ldexp(1.0, -l); /* cube side = leaf cell side, base units */
  double lo[3], hi[3];
  int64_t i0[3];
  for (int ax = 0; ax < 3; ++ax) {
    lo[ax] = t[ax] - 0.5 * s;
    hi[ax] = t[ax] + 0.5 * s;
    i0[ax] = (int64_t)floor(ldexp(lo[ax], l));
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 2; ++d) {
        int64_t P[3] = {i0[0] + a, i0[1] + b, i0[2] + d};
        double plo[3], phi[3];
        int empty = 0;
        for (int ax = 0; ax < 3; ++ax) {
          double clo = P[ax] * s;
          plo[ax] = lo[ax] > clo ? lo[ax] : clo;
          phi[ax] = hi[ax] < clo + s ? hi[ax] : clo + s;
          if (!(phi[ax] > plo[ax])) empty = 1;
        }
        if (!empty) visit_region(A, l, P[0], P[1], P[2], plo, phi, cb, ctx);
      }
}

typedef struct {
  double inv_cube;
} deposit_ctx;

static void deposit_cb(orc_amr* A, int l, long long c, double vol, void* ctx) {
  A->mass[l][c] += vol * ((deposit_ctx*)ctx)->inv_cube;
}

/* Mass assignment onto leaf cells, then coarse cell mass = sum of daughter
 * masses [Sec. 3.1]. Masses in units of the particle mass. */
void orc_amr_deposit(void* h) {
  orc_amr* A = (orc_amr*)h;
  for (int l = 0; l < A->nlev; ++l) memset(A->mass[l], 0, sizeof(double) * (size_t)A->ncell[l]);
  for (long long p = 0; p < A->Np; ++p) {
    const double* t = A->t + 3 * p;
    int l = leaf_level(A, t);
    deposit_ctx ctx = {ldexp(1.0, 3 * l)}; /* 1 / cube volume in base units */
    visit_particle(A, t, deposit_cb, &ctx);
  }
  for (int l = A->nlev - 1; l >= 1; --l) {
    int64_t Np = lev_dim(A, l - 1);
    for (long long o = 0; o < A->noct[l]; ++o) {
      int64_t key = A->keys[l][o];
      long long pc = find_cell(A, l - 1, key / (Np * Np), (key / Np) % Np, key % Np);
      double s = 0.0;
      for (int ch = 0; ch < 8; ++ch) s += A->mass[l][o * 8 + ch];
      A->mass[l - 1][pc] += s;
    }
  }
}

void orc_amr_masses(void* h, int l, double* out) {
  orc_amr* A = (orc_amr*)h;
  memcpy(out, A->mass[l], sizeof(double) * (size_t)A->ncell[l]);
}

/* delta per level: rho / rho_bar - 1 = m N_l^3 / Np - 1 (m in particle masses). */
void orc_amr_delta(void* h, int l, double* out) {
  orc_amr* A = (orc_amr*)h;
  double Nl = (double)lev_dim(A, l);
  double scale = Nl * Nl * Nl / (double)A->Np;
  for (long long c = 0; c < A->ncell[l]; ++c) out[c] = A->mass[l][c] * scale - 1.0;
}

/*
 * Mass of the solved hierarchy on a periodic PM grid of level lpm (N_pm =
 * N0 2^lpm) [Sec. 2.4, long-range part]: every leaf cell (a cell with no
 * daughters) carries a density contrast times its volume, and hands to each
 * PM cell it overlaps the fraction of that mass given by the overlapping
 * volume over its own.  The grids are nested, so a leaf either covers whole
 * PM cells (each receives its contrast as a density) or lies inside one
 * (which receives the contrast times 8^-(l - lpm)).  The contrast is
 *   what 0: delta_eff [Eq. (31)] (needs a model, orc_amr_set_model, and u);
 *   what 1: the matter contrast delta;
 *   what 2: delta + delta_eff, the right-hand side of Eq. (30).
 * out: N_pm^3 density contrasts (C order).
 */
void orc_amr_density_pm(void* h, int lpm, int what, double* out) {
  orc_amr* A = (orc_amr*)h;
  const orc_model* m = &A->model;
  const int64_t Npm = lev_dim(A, lpm);
  const double rho = m->omega_m / (m->a * m->a * m->a);
  for (long long q = 0; q < Npm * Npm * Npm; ++q) out[q] = 0.0;
  for (int l = 0; l < A->nlev; ++l) {
    const double Nl = (double)lev_dim(A, l);
    const double scale = Nl * Nl * Nl / (double)A->Np;
    for (long long c = 0; c < A->ncell[l]; ++c) {
      if (A->refined[l][c]) continue;
      const double d = A->mass[l][c] * scale - 1.0;
      double v = d;
      if (what != 1) {
        const double eff = d / 3.0 + m->Rt / (3.0 * rho) * (1.0 - exp(-A->u[l][c] / (m->n + 1)));
        v = what == 0 ? eff : d + eff;
      }
      int64_t I, J, K;
      cell_coords(A, l, c, &I, &J, &K);
      if (l <= lpm) {
        const int64_t sc = (int64_t)1 << (lpm - l);
        for (int64_t a = 0; a < sc; ++a)
          for (int64_t b = 0; b < sc; ++b)
            for (int64_t e = 0; e < sc; ++e)
              out[((I * sc + a) * Npm + (J * sc + b)) * Npm + (K * sc + e)] = v;
      } else {
        const int sh = l - lpm;
        out[((I >> sh) * Npm + (J >> sh)) * Npm + (K >> sh)] += v / (double)((int64_t)1 << (3 * sh));
      }
    }
  }
}

/* The effective mass alone (what 0 above). */
void orc_amr_effective_pm(void* h, int lpm, double* out) { orc_amr_density_pm(h, lpm, 0, out); }

/* Neighbour table of a level: nb[6c+d] >= 0 is a cell index, -1 a ghost.
 * Directions d: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z. */
static const int DIRS[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

/*
 * Value at level-l position (I,J,K) prolonged from the level-(l-1) field up
 * [Sec. 3.3, ghost cells]: parent value plus, per axis, s (c+ - c-)/8 when
 * both parent neighbours exist (else that component is 0).
 */
static double prolong_from_parent(const orc_amr* A, int l, const double* up, int64_t I, int64_t J,
                                  int64_t K, int linear) {
  int64_t P[3] = {(int64_t)floor(I / 2.0), (int64_t)floor(J / 2.0), (int64_t)floor(K / 2.0)};
  long long pc = find_cell(A, l - 1, P[0], P[1], P[2]);
  if (pc < 0) return NAN; /* cannot happen for hierarchies built above */
  double v = up[pc];
  if (!linear) return v;
  int64_t C[3] = {I, J, K};
  for (int ax = 0; ax < 3; ++ax) {
    int64_t Pp[3] = {P[0], P[1], P[2]}, Pm[3] = {P[0], P[1], P[2]};
    Pp[ax] += 1;
    Pm[ax] -= 1;
    long long cp = find_cell(A, l - 1, Pp[0], Pp[1], Pp[2]);
    long long cm = find_cell(A, l - 1, Pm[0], Pm[1], Pm[2]);
    if (cp < 0 || cm < 0) continue;
    double s = (wrapi(C[ax], lev_dim(A, l)) & 1) ? 1.0 : -1.0;
    v += s * (up[cp] - up[cm]) / 8.0;
  }
  return v;
}

typedef struct {
  long long n;
  long long* nb;    /* [6n] */
  double* ghost;    /* [6n] ghost u per (cell, direction) slot */
  unsigned char* colour;
} level_graph;

static void graph_build(const orc_amr* A, int l, level_graph* G, int linear) {
  long long n = A->ncell[l];
  G->n = n;
  G->nb = (long long*)malloc(sizeof(long long) * 6 * (size_t)n);
  G->ghost = (double*)calloc(6 * (size_t)n, sizeof(double));
  G->colour = (unsigned char*)malloc((size_t)n);
#pragma omp parallel for schedule(static) if (n >= 32768)
  for (long long c = 0; c < n; ++c) {
    int64_t I, J, K;
    cell_coords(A, l, c, &I, &J, &K);
    G->colour[c] = (unsigned char)((I + J + K) & 1);
    for (int d = 0; d < 6; ++d) {
      int64_t In = I + DIRS[d][0], Jn = J + DIRS[d][1], Kn = K + DIRS[d][2];
      long long nb = find_cell(A, l, In, Jn, Kn);
      G->nb[6 * c + d] = nb;
      if (nb < 0) G->ghost[6 * c + d] = prolong_from_parent(A, l, A->u[l - 1], In, Jn, Kn, linear);
    }
  }
}

static void graph_free(level_graph* G) {
  free(G->nb);
  free(G->ghost);
  free(G->colour);
}

static double graph_nb_u(const level_graph* G, const double* u, long long c, int d) {
  long long nb = G->nb[6 * c + d];
  return nb >= 0 ? u[nb] : G->ghost[6 * c + d];
}

/* L at cell c of a general level (ghosts as fixed neighbours) [Sec. 3.2]. */
static double graph_L(const level_graph* G, const double* u, long long c, double ih2,
                      const orc_model* m) {
  double uc = u[c], Ec = exp(uc), lap = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double um = graph_nb_u(G, u, c, 2 * ax), up = graph_nb_u(G, u, c, 2 * ax + 1);
    double bm = 0.5 * (exp(um) + Ec), bp = 0.5 * (exp(up) + Ec);
    lap += bm * um + bp * up - (bm + bp) * uc;
  }
  return lap * ih2 + m->alpha * m->Rt * (1.0 - exp(-uc / (m->n + 1)));
}

static double graph_dL(const level_graph* G, const double* u, long long c, double ih2,
                       const orc_model* m) {
  double uc = u[c], Ec = exp(uc), d = 0.0;
  for (int q = 0; q < 6; ++q) {
    double un = graph_nb_u(G, u, c, q);
    double b = 0.5 * (exp(un) + Ec);
    d += 0.5 * Ec * (un - uc) - b;
  }
  return d * ih2 + m->alpha * m->Rt / (m->n + 1) * exp(-uc / (m->n + 1));
}

static double graph_residual(const level_graph* G, const double* u, const double* f, double h,
                             const orc_model* m, double* r) {
  double ih2 = 1.0 / (h * h), s = 0.0;
  double* rr = r ? r : (double*)malloc(sizeof(double) * (size_t)G->n);
#pragma omp parallel for schedule(static) if (G->n >= 32768)
  for (long long c = 0; c < G->n; ++c) rr[c] = f[c] - graph_L(G, u, c, ih2, m);
  for (long long c = 0; c < G->n; ++c) s += rr[c] * rr[c];
  if (!r) free(rr);
  return sqrt(s);
}

static void graph_rb_sweep(const level_graph* G, double* u, const double* f, double h,
                           const orc_model* m, double step_cap) {
  double ih2 = 1.0 / (h * h);
  for (int colour = 0; colour < 2; ++colour)
#pragma omp parallel for schedule(static) if (G->n >= 32768)
    for (long long c = 0; c < G->n; ++c) {
      if (G->colour[c] != colour) continue;
      double step = (graph_L(G, u, c, ih2, m) - f[c]) / graph_dL(G, u, c, ih2, m);
      if (step > step_cap) step = step_cap;
      if (step < -step_cap) step = -step_cap;
      u[c] -= step;
    }
}

/* Source per level from the deposited masses (unless a custom one was set). */
static void amr_make_sources(orc_amr* A) {
  for (int l = 0; l < A->nlev; ++l) {
    if (A->f_custom[l]) continue;
    double Nl = (double)lev_dim(A, l);
    double scale = Nl * Nl * Nl / (double)A->Np;
    for (long long c = 0; c < A->ncell[l]; ++c)
      A->f[l][c] = A->model.src * (A->mass[l][c] * scale - 1.0);
  }
}

void orc_amr_set_model(void* h, double omega_m, double fr0_abs, int n, double a) {
  orc_amr* A = (orc_amr*)h;
  A->model = model_make(omega_m, fr0_abs, n, a);
  A->have_model = 1;
}

void orc_amr_set_source(void* h, int l, const double* f) {
  orc_amr* A = (orc_amr*)h;
  memcpy(A->f[l], f, sizeof(double) * (size_t)A->ncell[l]);
  A->f_custom[l] = 1;
}
void orc_amr_get_source(void* h, int l, double* out) {
  orc_amr* A = (orc_amr*)h;
  amr_make_sources(A);
  memcpy(out, A->f[l], sizeof(double) * (size_t)A->ncell[l]);
}
void orc_amr_set_u(void* h, int l, const double* u) {
  orc_amr* A = (orc_amr*)h;
  memcpy(A->u[l], u, sizeof(double) * (size_t)A->ncell[l]);
}
void orc_amr_get_u(void* h, int l, double* out) {
  orc_amr* A = (orc_amr*)h;
  memcpy(out, A->u[l], sizeof(double) * (size_t)A->ncell[l]);
}

/* Ghost values of level l (l >= 1) per (cell, direction) slot, NaN where the
 * neighbour exists. */
void orc_amr_ghosts(void* h, int l, int prolong_linear, double* out) {
  orc_amr* A = (orc_amr*)h;
  level_graph G;
  graph_build(A, l, &G, prolong_linear);
  for (long long q = 0; q < 6 * G.n; ++q) out[q] = G.nb[q] >= 0 ? NAN : G.ghost[q];
  graph_free(&G);
}

/* r = f - L(u) on level l with the current u of levels l and l-1. */
double orc_amr_residual(void* h, int l, int prolong_linear, double* r) {
  orc_amr* A = (orc_amr*)h;
  amr_make_sources(A);
  double hl = A->box / (double)lev_dim(A, l);
  if (l == 0) {
    dense_residual(A->u[0], A->f[0], A->N0, hl, &A->model, r);
    return norm2(r, A->ncell[0]);
  }
  level_graph G;
  graph_build(A, l, &G, prolong_linear);
  double rn = graph_residual(&G, A->u[l], A->f[l], hl, &A->model, r);
  graph_free(&G);
  return rn;
}

/*
 * r = f - L(u) at the given cells of level l only (ghost values prolonged from
 * the level l-1 field), for spot checks of large hierarchies [Sec. 3.2-3.3].
 */
void orc_amr_residual_at(void* h, int l, int prolong_linear, const long long* cells,
                         long long ncells, double* r) {
  orc_amr* A = (orc_amr*)h;
  amr_make_sources(A);
  const orc_model* m = &A->model;
  double hl = A->box / (double)lev_dim(A, l), ih2 = 1.0 / (hl * hl);
  for (long long q = 0; q < ncells; ++q) {
    long long c = cells[q];
    int64_t I, J, K;
    cell_coords(A, l, c, &I, &J, &K);
    double uc = A->u[l][c], Ec = exp(uc), lap = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
      double un[2];
      for (int s = 0; s < 2; ++s) {
        int d = 2 * ax + s;
        int64_t In = I + DIRS[d][0], Jn = J + DIRS[d][1], Kn = K + DIRS[d][2];
        long long nb = find_cell(A, l, In, Jn, Kn);
        un[s] = nb >= 0 ? A->u[l][nb]
                        : prolong_from_parent(A, l, A->u[l - 1], In, Jn, Kn, prolong_linear);
      }
      double bm = 0.5 * (exp(un[0]) + Ec), bp = 0.5 * (exp(un[1]) + Ec);
      lap += bm * un[0] + bp * un[1] - (bm + bp) * uc;
    }
    r[q] = A->f[l][c] - (lap * ih2 + m->alpha * m->Rt * (1.0 - exp(-uc / (m->n + 1))));
  }
}

/*
 * Solve refined level l >= 1 [Sec. 3.3, steps 9-10]: initial guess and ghost
 * values prolonged from level l-1; ghosts fixed; red-black NGS until
 * ||f - L(u)||_2 <= tol ||f||_2 over the level's cells.  If init_from_parent
 * is 0 the current u of the level is the initial guess.
 * out (nullable, 4 doubles): sweeps, ||r0||, ||r||, ||f||.
 */
int orc_amr_solve_level(void* h, int l, double tol, long long max_sweeps, int prolong_linear,
                        double step_cap, int init_from_parent, double* out) {
  orc_amr* A = (orc_amr*)h;
  amr_make_sources(A);
  double hl = A->box / (double)lev_dim(A, l);
  level_graph G;
  graph_build(A, l, &G, prolong_linear);
  if (init_from_parent) {
    for (long long c = 0; c < A->ncell[l]; ++c) {
      int64_t I, J, K;
      cell_coords(A, l, c, &I, &J, &K);
      A->u[l][c] = prolong_from_parent(A, l, A->u[l - 1], I, J, K, prolong_linear);
    }
  }
  double fn = norm2(A->f[l], A->ncell[l]);
  double r0 = graph_residual(&G, A->u[l], A->f[l], hl, &A->model, NULL);
  double target = tol * (fn > 0.0 ? fn : r0);
  double rn = r0;
  long long s = 0;
  while (rn > target && s < max_sweeps) {
    for (int q = 0; q < 10; ++q) graph_rb_sweep(&G, A->u[l], A->f[l], hl, &A->model, step_cap);
    s += 10;
    rn = graph_residual(&G, A->u[l], A->f[l], hl, &A->model, NULL);
  }
  graph_free(&G);
  if (out) {
    out[0] = (double)s;
    out[1] = r0;
    out[2] = rn;
    out[3] = fn;
  }
  return rn <= target ? 0 : 1;
}

/*
 * Full one-way solve [Sec. 3.3, steps 1-12]: base level by FAS V-cycles from
 * u0_base (nullable -> zero), then each refined level in turn.
 * stats (nullable, 4 + 4*nlev doubles): [0] base V-cycles, [1] base ||r||/||f||,
 * [2] converged flag (all levels), then per level l >= 1 the
 * orc_amr_solve_level outputs at [4 + 4(l-1) ...].
 */
int orc_amr_solve(void* h, double tol, int max_vcycles, long long max_sweeps_refined, int n_pre,
                  int n_post, int prolong_linear, double step_cap, const double* u0_base,
                  double* stats) {
  orc_amr* A = (orc_amr*)h;
  amr_make_sources(A);
  long long nb = A->ncell[0];
  if (u0_base) memcpy(A->u[0], u0_base, sizeof(double) * (size_t)nb);
  else memset(A->u[0], 0, sizeof(double) * (size_t)nb);
  double st[8];
  int bad = orc_solve_dense_f(A->N0, A->box, A->f[0], A->model.omega_m, A->model.fr0_abs,
                              A->model.n, A->model.a,
                              A->u[0], tol, max_vcycles, n_pre, n_post, prolong_linear, step_cap,
                              st) != 0;
  if (stats) {
    stats[0] = st[0];
    stats[1] = st[4] > 0 ? st[2] / st[4] : st[2];
    stats[3] = st[5];
  }
  for (int l = 1; l < A->nlev; ++l) {
    double o[4];
    bad |= orc_amr_solve_level(h, l, tol, max_sweeps_refined, prolong_linear, step_cap, 1, o) != 0;
    if (stats) for (int q = 0; q < 4; ++q) stats[4 + 4 * (l - 1) + q] = o[q];
  }
  if (stats) stats[2] = bad ? 0.0 : 1.0;
  return bad;
}

/*
 * f_R and a_MG / c^2 = grad_x f_R / (2a) per level [Sec. 2, Eq. (13)];
 * central differences with ghost values at patch edges.  acc: [ncell][3].
 */
void orc_amr_level_force(void* h, int l, int prolong_linear, double* fr, double* acc) {
  orc_amr* A = (orc_amr*)h;
  const orc_model* m = &A->model;
  long long n = A->ncell[l];
  double hl = A->box / (double)lev_dim(A, l);
  for (long long c = 0; c < n; ++c) fr[c] = m->fbar * exp(A->u[l][c]);
  if (!acc) return;
  if (l == 0) {
    int N = A->N0;
    double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* frt = (double*)malloc(sizeof(double) * (size_t)n);
    orc_force_dense(N, A->box, m->omega_m, m->fr0_abs, m->n, m->a, A->u[0], frt, tmp);
    for (long long c = 0; c < n; ++c)
      for (int ax = 0; ax < 3; ++ax) acc[3 * c + ax] = tmp[ax * n + c];
    free(tmp);
    free(frt);
    return;
  }
  level_graph G;
  graph_build(A, l, &G, prolong_linear);
  for (long long c = 0; c < n; ++c) {
    for (int ax = 0; ax < 3; ++ax) {
      double um = graph_nb_u(&G, A->u[l], c, 2 * ax), up = graph_nb_u(&G, A->u[l], c, 2 * ax + 1);
      double g = (m->fbar * exp(up) - m->fbar * exp(um)) / (2.0 * hl);
      acc[3 * c + ax] = g / (2.0 * m->a);
    }
  }
  graph_free(&G);
}

typedef struct {
  double inv_cube;
  double* accl[ORC_MAXLEV];
  double out[3];
} gather_ctx;

static void gather_cb(orc_amr* A, int l, long long c, double vol, void* ctx) {
  (void)A;
  gather_ctx* g = (gather_ctx*)ctx;
  double w = vol * g->inv_cube;
  for (int ax = 0; ax < 3; ++ax) g->out[ax] += w * g->accl[l][3 * c + ax];
}

/* Force at the particles: the leaf-cell values gathered with the same
 * overlap weights as the mass assignment (adjoint of the deposit).
 * acc: [Np][3]. */
void orc_amr_particle_force(void* h, int prolong_linear, double* acc) {
  orc_amr* A = (orc_amr*)h;
  gather_ctx g;
  memset(&g, 0, sizeof(g));
  for (int l = 0; l < A->nlev; ++l) {
    double* fr = (double*)malloc(sizeof(double) * (size_t)A->ncell[l]);
    g.accl[l] = (double*)malloc(sizeof(double) * 3 * (size_t)A->ncell[l]);
    orc_amr_level_force(h, l, prolong_linear, fr, g.accl[l]);
    free(fr);
  }
  for (long long p = 0; p < A->Np; ++p) {
    const double* t = A->t + 3 * p;
    int l = leaf_level(A, t);
    g.inv_cube = ldexp(1.0, 3 * l);
    g.out[0] = g.out[1] = g.out[2] = 0.0;
    visit_particle(A, t, gather_cb, &g);
    for (int ax = 0; ax < 3; ++ax) acc[3 * p + ax] = g.out[ax];
  }
  for (int l = 0; l < A->nlev; ++l) free(g.accl[l]);
}

/* Leaf level of each particle (for structure checks). */
void orc_amr_particle_levels(void* h, int* out) {
  orc_amr* A = (orc_amr*)h;
  for (long long p = 0; p < A->Np; ++p) out[p] = leaf_level(A, A->t + 3 * p);
}
