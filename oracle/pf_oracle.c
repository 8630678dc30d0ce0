/*
 * pf_oracle.c -- plain, slow FP64 CPU oracle of the Poisson-Fermi solver
 * (Chen, Chen, Liu, "A GPU Poisson-Fermi Solver for Ion Channel Simulations").
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU-baseline
 * leg of the benchmark; never by the product path.  Every function follows one
 * passage of the paper, cited beside it, in the paper's order and notation, with no
 * blocking, fusion or reordering.  Readings of passages the paper leaves open:
 *   - by default charges are spread trilinearly onto the grid instead of the Green's-
 *     function decomposition of Eqs. (5)-(10), so the SMIB interface rows of Eqs. (17)-(18)
 *     carry no jump term and reduce to harmonic-mean face coefficients; the decomposition
 *     itself (pfo_decompose, charge_mode 1) takes phi^L = -phi* on the interface and the
 *     jump of Eq. (8), the signs that keep phi continuous (Eqs. 10 and 16 print others);
 *   - conjugate gradients (pfo_pcg) run in the inner product that weights a node by 1/2
 *     per mirrored side, in which the stored operators are symmetric;
 *   - the filter region of Eqs. (19)-(20) is a node mask of Dirichlet values for the
 *     continuum solves (pfo_pf_solve_fixed), with the six site points at +-a along the axes;
 *   - Gamma in Eq. (1) is taken from its own definition (an implicit pointwise
 *     equation) rather than lagged from the previous iterate;
 *   - Psi = 0 (Eq. 14) at membrane nodes and on the Dirichlet planes; the x/y sides
 *     keep the zero-flux mirror of Eq. (4);
 *   - the fixed charges enter the PF2 right-hand side at whatever node type holds them;
 *   - Jacobi preconditioning is the right-preconditioned form of BiCGSTAB.
 * The OpenMP pragmas are inert in the checker build (compiled without -fopenmp); only the
 * benchmark's all-cores timing copy of this file is compiled with them.
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Table 1 constants ---------------------------------------------------- */
static const double KB = 1.38e-23;        /* J/K */
static const double QE = 1.602e-19;       /* C */
static const double EPS0 = 8.85e-12;      /* F/m  (8.85e-14 F/cm) */
static const double NAVO = 6.02214076e23; /* 1/mol; not printed in the paper (CODATA) */

double pfo_thermal_voltage(double T) { return KB * T / QE; }

/* e^2/(eps0 k_B T) expressed in Angstrom: the factor that turns -div(eps eps0 grad phi)
 * = sum q C into -div(eps grad phi_hat) = lambda * sum z C with C in A^-3. */
double pfo_lambda(double T) { return QE * QE / (EPS0 * KB * T * 1e-10); }

double pfo_molar_to_per_A3(void) { return NAVO * 1e-27; }

/* ---- species: Eq. (1) definitions of v_i, v_0, Gamma^B ----------------------- */
int pfo_species_setup(int ns, const double* z, const double* radius_A, const double* bulk_M,
                      double* v, double* p, double* cB, double* gammaB) {
  if (ns < 1) return PFO_E_INVAL;
  double v0 = 0.0;
  for (int i = 0; i < ns; ++i) {
    if (radius_A[i] <= 0.0 || bulk_M[i] < 0.0) return PFO_E_INVAL;
    v[i] = 4.0 * M_PI * radius_A[i] * radius_A[i] * radius_A[i] / 3.0;
    v0 += v[i];
  }
  v0 /= ns; /* average volume over the K ions and water */
  double g = 1.0, charge = 0.0, scale = 0.0;
  for (int i = 0; i < ns; ++i) {
    p[i] = v[i] / v0;
    cB[i] = bulk_M[i] * pfo_molar_to_per_A3();
    g -= v[i] * cB[i];
    charge += z[i] * cB[i];
    scale += fabs(z[i]) * cB[i];
  }
  *gammaB = g;
  if (g <= 0.0) return PFO_E_INVAL;
  if (fabs(charge) > 1e-12 * (scale > 0.0 ? scale : 1.0)) return PFO_E_INVAL; /* neutral bath */
  return PFO_OK;
}

/* ---- Eq. (1): Fermi-like concentrations and steric potential ----------------
 * With C_i = cB_i exp(-z_i phi + p_i S), S = ln(Gamma/GammaB) and Gamma = 1 - sum v_i C_i,
 * Gamma is the root of  f(u) = e^u + sum_i exp(la_i + p_i u) - 1,  u = ln Gamma,
 * la_i = ln(v_i cB_i) - z_i phi - p_i ln GammaB.  f is increasing, so the root is unique. */
int pfo_fermi_point(int ns, const double* z, const double* v, const double* p, const double* cB,
                    double gammaB, double phi_hat, double* C, double* S, double* Gamma, int* iters) {
  double la[64];
  int used[64];
  if (ns > 64) return PFO_E_INVAL;
  const double lgB = log(gammaB);
  int nterm = 0;
  for (int i = 0; i < ns; ++i) {
    used[i] = (cB[i] > 0.0);
    if (used[i]) {
      la[i] = log(v[i] * cB[i]) - z[i] * phi_hat - p[i] * lgB;
      ++nterm;
    }
  }
  /* bracket: at u_hi some term (or e^u) reaches 1, so f > 0; at u_lo every one of the
   * nterm+1 positive parts is at most 1/(nterm+1), so f <= 0. */
  const double lnn = log((double)(nterm + 1));
  double hi = 0.0, lo = -lnn;
  for (int i = 0; i < ns; ++i) {
    if (!used[i]) continue;
    double a = -la[i] / p[i];
    double b = (-la[i] - lnn) / p[i];
    if (a < hi) hi = a;
    if (b < lo) lo = b;
  }
  double u = lgB;
  if (!(u < hi && u > lo)) u = 0.5 * (lo + hi);
  int it = 0, ok = 0;
  for (it = 1; it <= 400; ++it) {
    double f = exp(u) - 1.0, df = exp(u);
    for (int i = 0; i < ns; ++i) {
      if (!used[i]) continue;
      double term = exp(la[i] + p[i] * u);
      f += term;
      df += p[i] * term;
    }
    if (f == 0.0) { ok = 1; break; }
    if (f > 0.0) hi = u; else lo = u;
    double un = u - f / df;
    if (!(un > lo && un < hi)) un = 0.5 * (lo + hi); /* safeguard: bisect */
    double du = un - u;
    u = un;
    if (fabs(du) <= 1e-15 * (fabs(u) > 1.0 ? fabs(u) : 1.0)) { ok = 1; break; }
  }
  if (iters) *iters = it;
  if (!ok || !isfinite(u)) return PFO_E_GAMMA;
  const double s = u - lgB;
  for (int i = 0; i < ns; ++i)
    C[i] = used[i] ? exp(log(cB[i]) - z[i] * phi_hat + p[i] * s) : 0.0;
  *S = s;
  *Gamma = exp(u);
  return PFO_OK;
}

/* ---- 7-point FD operators in the diagonal storage of Section 4 --------------- */
/* Eq. (1) at n nodes, one after another (the pointwise step of the Table 2 loop over a node list):
 * C (species-major, n per species) in A^-3, S and Gamma; PFO_OK, or the largest status of a node that failed. */
int pfo_fermi_nodes(int ns, const double* z, const double* v, const double* p, const double* cB, double gammaB,
                    long n, const double* phi_hat, double* C, double* S, double* Gamma) {
  int status = PFO_OK;
  if (ns < 1 || ns > 64) return PFO_E_INVAL;
#pragma omp parallel for schedule(static) reduction(max : status)
  for (long c = 0; c < n; ++c) {
    double Ci[64], s, g;
    const int st = pfo_fermi_point(ns, z, v, p, cB, gammaB, phi_hat[c], Ci, &s, &g, NULL);
    if (st > status) status = st;
    for (int i = 0; i < ns; ++i) C[(long)i * n + c] = Ci[i];
    S[c] = s;
    Gamma[c] = g;
  }
  return status;
}

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* Eqs. (7), (13), (15)-(18): with a zero jump the SMIB rows at x_l, x_{l+1} are
 * eps_m[-phi_{l-1} + (2-c1) phi_l - c2 phi_{l+1}] and eps_s[-d1 phi_l + (2-d2) phi_{l+1} - phi_{l+2}],
 * i.e. the flux form with face coefficient eps_m c2 = eps_s d1 = 2 eps_m eps_s/(eps_m+eps_s). */
int pfo_assemble_eps(int nx, int ny, int nz, double h, const double* eps, const double* sigma,
                     double* A) {
  if (nx < 2 || ny < 2 || nz < 3 || h <= 0.0) return PFO_E_INVAL;
  const long N = (long)nx * ny * nz, sx = 1, sy = nx, sz = (long)nx * ny;
  const double ih2 = 1.0 / (h * h);
  memset(A, 0, sizeof(double) * 7 * N);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long c = i + nx * ((long)j + (long)ny * k);
        if (k == 0 || k == nz - 1) { A[c] = 1.0; continue; } /* Dirichlet row, Eq. (4) */
        const double e = eps[c];
        double diag = 0.0, w;
        /* east / west; at a side the ghost node mirrors its inner neighbour (zero flux) */
        if (i < nx - 1) { w = harmonic(e, eps[c + sx]) * ih2; A[1 * N + c] -= w; diag += w; }
        else            { w = harmonic(e, eps[c - sx]) * ih2; A[2 * N + c] -= w; diag += w; }
        if (i > 0)      { w = harmonic(e, eps[c - sx]) * ih2; A[2 * N + c] -= w; diag += w; }
        else            { w = harmonic(e, eps[c + sx]) * ih2; A[1 * N + c] -= w; diag += w; }
        /* north / south */
        if (j < ny - 1) { w = harmonic(e, eps[c + sy]) * ih2; A[4 * N + c] -= w; diag += w; }
        else            { w = harmonic(e, eps[c - sy]) * ih2; A[3 * N + c] -= w; diag += w; }
        if (j > 0)      { w = harmonic(e, eps[c - sy]) * ih2; A[3 * N + c] -= w; diag += w; }
        else            { w = harmonic(e, eps[c + sy]) * ih2; A[4 * N + c] -= w; diag += w; }
        /* up / down: interior planes always have both neighbours */
        w = harmonic(e, eps[c + sz]) * ih2; A[6 * N + c] -= w; diag += w;
        w = harmonic(e, eps[c - sz]) * ih2; A[5 * N + c] -= w; diag += w;
        A[c] = diag + (sigma ? sigma[c] : 0.0);
      }
  return PFO_OK;
}

/* Eqs. (12), (14): eps_s (lc^2 Lap - 1) Psi = rho, written as eps_s lc^2 (-Lap_h) Psi + eps_s Psi
 * = -rho; Psi = 0 on the boundary of the solvent domain. */
int pfo_assemble_pf1(int nx, int ny, int nz, double h, const unsigned char* solvent,
                     double eps_s, double lc, double* A) {
  if (nx < 2 || ny < 2 || nz < 3 || h <= 0.0) return PFO_E_INVAL;
  const long N = (long)nx * ny * nz;
  const double w = eps_s * lc * lc / (h * h);
  memset(A, 0, sizeof(double) * 7 * N);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long c = i + nx * ((long)j + (long)ny * k);
        if (k == 0 || k == nz - 1 || !solvent[c]) { A[c] = 1.0; continue; }
        if (i < nx - 1) A[1 * N + c] -= w; else A[2 * N + c] -= w;
        if (i > 0) A[2 * N + c] -= w; else A[1 * N + c] -= w;
        if (j < ny - 1) A[4 * N + c] -= w; else A[3 * N + c] -= w;
        if (j > 0) A[3 * N + c] -= w; else A[4 * N + c] -= w;
        A[6 * N + c] -= w;
        A[5 * N + c] -= w;
        A[c] = 6.0 * w + eps_s;
      }
  return PFO_OK;
}

void pfo_dia_apply(int nx, int ny, int nz, const double* A, const double* x, double* y) {
  const long N = (long)nx * ny * nz, sy = nx, sz = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long c = i + nx * ((long)j + (long)ny * k);
        double s = A[c] * x[c];
        if (i < nx - 1) s += A[1 * N + c] * x[c + 1];
        if (i > 0) s += A[2 * N + c] * x[c - 1];
        if (j > 0) s += A[3 * N + c] * x[c - sy];
        if (j < ny - 1) s += A[4 * N + c] * x[c + sy];
        if (k > 0) s += A[5 * N + c] * x[c - sz];
        if (k < nz - 1) s += A[6 * N + c] * x[c + sz];
        y[c] = s;
      }
}

static double dot(long n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double norm_inf(long n, const double* a) {
  double m = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m)
  for (long i = 0; i < n; ++i) if (fabs(a[i]) > m) m = fabs(a[i]);
  return m;
}

static int is_identity_row(long N, const double* A, long c) {
  if (A[c] != 1.0) return 0;
  for (int d = 1; d < 7; ++d) if (A[d * N + c] != 0.0) return 0;
  return 1;
}

/* Table 3 (GPU Algorithm 1) with the Jacobi preconditioner M = diag(A) applied from the
 * right, as in the preconditioned BiCGSTAB of the Templates book that the paper cites. */
int pfo_bicgstab(int nx, int ny, int nz, const double* A, const double* b, double* x,
                 int max_it, double tol, int norm_mode, int* iters, double* res) {
  const long N = (long)nx * ny * nz;
  double* r = malloc(sizeof(double) * N);
  double* rt = malloc(sizeof(double) * N);
  double* p = malloc(sizeof(double) * N);
  double* ph = malloc(sizeof(double) * N);
  double* v = malloc(sizeof(double) * N);
  double* s = malloc(sizeof(double) * N);
  double* sh = malloc(sizeof(double) * N);
  double* t = malloc(sizeof(double) * N);
  int status = PFO_E_NOCONV, it = 0;
  double measure = 0.0;
  if (!r || !rt || !p || !ph || !v || !s || !sh || !t) { status = PFO_E_INVAL; goto done; }

  for (long c = 0; c < N; ++c) if (is_identity_row(N, A, c)) x[c] = b[c];

  double bnorm = sqrt(dot(N, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
#define PFO_MEASURE(vec) (norm_mode == 0 ? sqrt(dot(N, vec, vec)) / bnorm : norm_inf(N, vec))
#define PFO_CONVERGED(m) (norm_mode == 0 ? (m) <= tol : (m) < tol)

  pfo_dia_apply(nx, ny, nz, A, x, r); /* r0 = b - A x0; the shadow residual rtilde = r0 */
  for (long c = 0; c < N; ++c) { r[c] = b[c] - r[c]; rt[c] = r[c]; }
  measure = PFO_MEASURE(r);
  if (PFO_CONVERGED(measure)) { status = PFO_OK; goto done; }

  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (it = 1; it <= max_it; ++it) {
    const double rho = dot(N, rt, r); /* rho = rtilde . r */
    if (rho == 0.0) { status = PFO_E_BREAKDOWN; break; }
    if (it == 1) {
#pragma omp parallel for schedule(static)
      for (long c = 0; c < N; ++c) p[c] = r[c]; /* first direction p = r */
    } else {
      const double beta = (rho / rho_prev) * (alpha / omega);
#pragma omp parallel for schedule(static)
      for (long c = 0; c < N; ++c) p[c] = r[c] + beta * (p[c] - omega * v[c]);
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) ph[c] = p[c] / A[c]; /* Jacobi: phat = M^-1 p */
    pfo_dia_apply(nx, ny, nz, A, ph, v); /* v = A phat */
    const double rtv = dot(N, rt, v);
    if (rtv == 0.0) { status = PFO_E_BREAKDOWN; break; }
    alpha = rho / rtv;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) s[c] = r[c] - alpha * v[c];
    measure = PFO_MEASURE(s);
    if (PFO_CONVERGED(measure)) { /* early exit on s: x = x + alpha phat */
      for (long c = 0; c < N; ++c) x[c] += alpha * ph[c];
      status = PFO_OK;
      break;
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) sh[c] = s[c] / A[c];
    pfo_dia_apply(nx, ny, nz, A, sh, t); /* t = A shat */
    const double tt = dot(N, t, t);
    if (tt == 0.0) { status = PFO_E_BREAKDOWN; break; }
    omega = dot(N, t, s) / tt; /* minimises ||s - omega t||_2 */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) x[c] += alpha * ph[c] + omega * sh[c];
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) r[c] = s[c] - omega * t[c];
    measure = PFO_MEASURE(r);
    if (PFO_CONVERGED(measure)) { status = PFO_OK; break; }
    if (omega == 0.0) { status = PFO_E_BREAKDOWN; break; }
    rho_prev = rho;
  }
  if (it > max_it) it = max_it;
#undef PFO_MEASURE
#undef PFO_CONVERGED
done:
  if (iters) *iters = it;
  if (res) *res = measure;
  free(r); free(rt); free(p); free(ph); free(v); free(s); free(sh); free(t);
  return status;
}

/* Conjugate gradients for the systems the paper calls symmetric (Section 3: the Laplace
 * equation (9) and PF1 (12)).  The 7-diagonal operators here keep identity rows for fixed
 * nodes and mirror ghosts on the x/y sides, so A itself is not symmetric: a mirror doubles a side
 * row's coupling to its inner neighbour.  Weighting each row by w = (1/2 per mirrored direction)
 * gives W A symmetric on the rows that are not identity rows, and with x = b on the identity rows
 * the residual and every search direction vanish there.  Conjugate gradients in the inner product
 * <u, v>_W = sum_c w_c u_c v_c with the Jacobi preconditioner M = diag(A) (a diagonal, hence
 * self-adjoint in that inner product) is then ordinary preconditioned CG on W A x = W b. */
static double side_weight(int nx, int ny, long c) {
  const long i = c % nx, j = (c / nx) % ny;
  return (i == 0 || i == nx - 1 ? 0.5 : 1.0) * (j == 0 || j == ny - 1 ? 0.5 : 1.0);
}

/* Largest |w_c A_cn - w_n A_nc| over couplings between rows that are not identity rows, relative
 * to the largest |w_c A_cn|.  Zero (to rounding) for the operators of pfo_assemble_eps and
 * pfo_assemble_pf1. */
double pfo_weighted_asymmetry(int nx, int ny, int nz, const double* A) {
  const long N = (long)nx * ny * nz, sy = nx, sz = (long)nx * ny;
  double worst = 0.0, scale = 0.0;
  for (long c = 0; c < N; ++c) {
    if (is_identity_row(N, A, c)) continue;
    const long i = c % nx, j = (c / nx) % ny, k = c / sz;
    /* (diagonal slot of the neighbour, its slot pointing back, offset) */
    const int fwd[6] = {1, 2, 3, 4, 5, 6}, back[6] = {2, 1, 4, 3, 6, 5};
    const long off[6] = {1, -1, -sy, sy, -sz, sz};
    const int ok[6] = {i < nx - 1, i > 0, j > 0, j < ny - 1, k > 0, k < nz - 1};
    for (int d = 0; d < 6; ++d) {
      if (!ok[d]) continue;
      const long n = c + off[d];
      if (is_identity_row(N, A, n)) continue;
      const double a = side_weight(nx, ny, c) * A[fwd[d] * N + c];
      const double b = side_weight(nx, ny, n) * A[back[d] * N + n];
      if (fabs(a) > scale) scale = fabs(a);
      if (fabs(a - b) > worst) worst = fabs(a - b);
    }
  }
  return scale > 0.0 ? worst / scale : 0.0;
}

static double wdot(int nx, int ny, long n, const double* a, const double* b) {
  double s = 0.0;
  for (long c = 0; c < n; ++c) s += side_weight(nx, ny, c) * a[c] * b[c];
  return s;
}

int pfo_pcg(int nx, int ny, int nz, const double* A, const double* b, double* x,
            int max_it, double tol, int norm_mode, int* iters, double* res) {
  const long N = (long)nx * ny * nz;
  double* r = malloc(sizeof(double) * N);
  double* z = malloc(sizeof(double) * N);
  double* p = malloc(sizeof(double) * N);
  double* q = malloc(sizeof(double) * N);
  int status = PFO_E_NOCONV, it = 0;
  double measure = 0.0;
  if (!r || !z || !p || !q) { status = PFO_E_INVAL; goto done; }
  for (long c = 0; c < N; ++c)
    if (!(A[c] > 0.0)) { status = PFO_E_INVAL; goto done; } /* M = diag(A) must be positive */
  if (pfo_weighted_asymmetry(nx, ny, nz, A) > 1e-13) { status = PFO_E_INVAL; goto done; }

  for (long c = 0; c < N; ++c) if (is_identity_row(N, A, c)) x[c] = b[c];
  double bnorm = sqrt(dot(N, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
#define PFO_MEASURE(vec) (norm_mode == 0 ? sqrt(dot(N, vec, vec)) / bnorm : norm_inf(N, vec))
#define PFO_CONVERGED(m) (norm_mode == 0 ? (m) <= tol : (m) < tol)

  pfo_dia_apply(nx, ny, nz, A, x, r); /* r = b - A x */
  for (long c = 0; c < N; ++c) r[c] = b[c] - r[c];
  measure = PFO_MEASURE(r);
  if (PFO_CONVERGED(measure)) { status = PFO_OK; goto done; }
  for (long c = 0; c < N; ++c) { z[c] = r[c] / A[c]; p[c] = z[c]; } /* z = M^-1 r, p = z */
  double rz = wdot(nx, ny, N, r, z);
  for (it = 1; it <= max_it; ++it) {
    pfo_dia_apply(nx, ny, nz, A, p, q); /* q = A p */
    const double pq = wdot(nx, ny, N, p, q);
    if (!(pq > 0.0)) { status = PFO_E_BREAKDOWN; break; } /* not positive definite */
    const double alpha = rz / pq;
    for (long c = 0; c < N; ++c) { x[c] += alpha * p[c]; r[c] -= alpha * q[c]; }
    measure = PFO_MEASURE(r);
    if (PFO_CONVERGED(measure)) { status = PFO_OK; break; }
    for (long c = 0; c < N; ++c) z[c] = r[c] / A[c];
    const double rz_next = wdot(nx, ny, N, r, z);
    const double beta = rz_next / rz;
    for (long c = 0; c < N; ++c) p[c] = z[c] + beta * p[c];
    rz = rz_next;
  }
  if (it > max_it) it = max_it;
#undef PFO_MEASURE
#undef PFO_CONVERGED
done:
  if (iters) *iters = it;
  if (res) *res = measure;
  free(r); free(z); free(p); free(q);
  return status;
}

/* Eq. (3) with the point charges spread onto the grid by trilinear weights: the source
 * lambda * q_j * delta(r - r_j) becomes lambda q_j w_c / h^3 at the 8 corners c. */
int pfo_spread_charges(int nx, int ny, int nz, double h, const double* origin, int nq,
                       const double* charges, double lambda, double* f) {
  const int n[3] = {nx, ny, nz};
  for (int q = 0; q < nq; ++q) {
    int i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
      const double g = (charges[4 * q + a] - origin[a]) / h;
      int i = (int)floor(g);
      if (i == n[a] - 1 && g == (double)(n[a] - 1)) i = n[a] - 2; /* on the last plane */
      if (!(g >= 0.0) || i < 0 || i > n[a] - 2) return PFO_E_INVAL;
      i0[a] = i;
      t[a] = g - i;
    }
    const double amp = lambda * charges[4 * q + 3] / (h * h * h);
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
      const double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
      const long id = (i0[0] + dx) + (long)nx * ((i0[1] + dy) + (long)ny * (i0[2] + dz));
      f[id] += amp * w;
    }
  }
  return PFO_OK;
}

/* ---- Table 2: the sequential PF nonlinear solver (initial PF2 solve, then PF1, PF2 and the
 * relaxation until the update is small; the charges are spread onto the grid, so no singular part
 * is split off) ----------------------------------------------------------------- */
/* ---- potential decomposition (Eqs. 5-10) and the interface right-hand side (Eqs. 8, 16-18) ----
 *
 * In the biomolecular region Omega_m (the non-solvent nodes) the potential is split as
 * phi = phi~ + G with G = phi* + phi^L:  phi* is the Coulomb potential of the point charges in a
 * uniform dielectric eps_m (in scaled units lambda q / (4 pi eps_m |r - r_j|)), and phi^L is harmonic
 * in Omega_m (Eq. 9) with G = 0 on the interface with the solvent, i.e. phi^L = -phi* there (Eq. 10
 * read with the sign that keeps phi continuous), and with zero normal derivative of G on the x/y box
 * sides (the zero-flux sides of Eq. 4).  phi~ then has no singular source, is continuous, and its flux
 * jumps by eps_m dG/dn across the interface (Eq. 8, n from Omega_m to Omega_s).  With the interface at
 * the midpoint of each face between a membrane and a solvent node, the SMIB rows (17)-(18) are the
 * harmonic-face rows plus c0/h^2 on the membrane row and d0/h^2 on the solvent row, with
 * c0 = -eps_m h J / (eps_m + eps_s), d0 = -eps_s h J / (eps_m + eps_s), J = eps_m dG/dn at the midpoint. */
static void coulomb(int nq, const double* ch, double coef, const double r[3], double* phi, double grad[3]) {
  double p = 0.0, g[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < nq; ++j) {
    const double d[3] = {r[0] - ch[4 * j], r[1] - ch[4 * j + 1], r[2] - ch[4 * j + 2]};
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double inv = 1.0 / sqrt(d2);
    const double qj = ch[4 * j + 3];
    p += qj * inv;
    for (int a = 0; a < 3; ++a) g[a] -= qj * d[a] * inv * inv * inv;
  }
  if (phi) *phi = coef * p;
  if (grad)
    for (int a = 0; a < 3; ++a) grad[a] = coef * g[a];
}

int pfo_decompose(int nx, int ny, int nz, double h, const double* origin, const unsigned char* solvent,
                  int nq, const double* charges, double eps_m, double eps_s, double lambda, double* G,
                  double* bif, int* lin_iters) {
  if (nx < 3 || ny < 3 || nz < 3 || h <= 0.0 || eps_m <= 0.0 || eps_s <= 0.0 || nq < 0) return PFO_E_INVAL;
  const long N = (long)nx * ny * nz;
  const int n3[3] = {nx, ny, nz};
  const long st3[3] = {1, nx, (long)nx * ny};
  const double coef = lambda / (4.0 * M_PI * eps_m);
  /* charges strictly inside the box and off the nodes (G is evaluated at nodes) */
  for (int j = 0; j < nq; ++j)
    for (int a = 0; a < 3; ++a) {
      const double g = (charges[4 * j + a] - origin[a]) / h;
      if (!(g > 0.0 && g < n3[a] - 1)) return PFO_E_INVAL;
    }
  for (long c = 0; c < N; ++c) {
    const int i = (int)(c % nx), jj = (int)((c / nx) % ny);
    const double r[3] = {origin[0] + h * i, origin[1] + h * jj, origin[2] + h * (double)(c / ((long)nx * ny))};
    for (int j = 0; j < nq; ++j) {
      const double d2 = (r[0] - charges[4 * j]) * (r[0] - charges[4 * j]) +
                        (r[1] - charges[4 * j + 1]) * (r[1] - charges[4 * j + 1]) +
                        (r[2] - charges[4 * j + 2]) * (r[2] - charges[4 * j + 2]);
      if (d2 < 1e-12 * h * h) return PFO_E_INVAL;
    }
    /* a side node and its mirror partner must be of the same kind (no interface across a mirror) */
    if ((i == 0 && solvent[c] != solvent[c + 1]) || (i == nx - 1 && solvent[c] != solvent[c - 1]) ||
        (jj == 0 && solvent[c] != solvent[c + nx]) || (jj == ny - 1 && solvent[c] != solvent[c - nx]))
      return PFO_E_INVAL;
  }
  double* A = calloc((size_t)7 * N, sizeof(double));
  double* b = calloc(N, sizeof(double));
  double* phiL = calloc(N, sizeof(double));
  int status = PFO_OK;
  if (!A || !b || !phiL) { status = PFO_E_INVAL; goto out; }

  /* phi^L: -Lap_h phi^L = 0 at membrane nodes off the Dirichlet planes, Shortley-Weller differences to
   * the interface midpoints (distance h/2, value -phi*), zero normal derivative of G on the x/y sides */
  for (long c = 0; c < N; ++c) {
    const long k = c / ((long)nx * ny);
    const int idx[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)k};
    const double r[3] = {origin[0] + h * idx[0], origin[1] + h * idx[1], origin[2] + h * idx[2]};
    if (solvent[c] || k == 0 || k == nz - 1) {
      A[c] = 1.0;
      if (!solvent[c]) { double p; coulomb(nq, charges, coef, r, &p, NULL); b[c] = -p; } /* G = 0 on the planes */
      continue;
    }
    for (int a = 0; a < 3; ++a) {
      /* diagonal slots of the neighbour below / above along axis a: west, south, down / east, north, up */
      const int slot_of[2] = {a == 0 ? 2 : a == 1 ? 3 : 5, a == 0 ? 1 : a == 1 ? 4 : 6};
      if (a < 2 && (idx[a] == 0 || idx[a] == n3[a] - 1)) {
        /* box side: dG/dn = 0, so the ghost value is partner + 2h dphi^L/dn = partner - 2h dphi_star/dn */
        const int low = idx[a] == 0;
        double gr[3];
        coulomb(nq, charges, coef, r, NULL, gr);
        const double nout = low ? -1.0 : 1.0;
        A[c] += 2.0 / (h * h);
        A[slot_of[low ? 1 : 0] * N + c] -= 2.0 / (h * h);
        b[c] += -2.0 * nout * gr[a] / h;
        continue;
      }
      double hs[2], val[2];
      int bnd[2];
      for (int sgn = 0; sgn < 2; ++sgn) {
        const long nb = c + (sgn ? st3[a] : -st3[a]);
        if (solvent[nb]) {
          double rx[3] = {r[0], r[1], r[2]};
          rx[a] += (sgn ? 0.5 : -0.5) * h;
          double p;
          coulomb(nq, charges, coef, rx, &p, NULL);
          hs[sgn] = 0.5 * h;
          val[sgn] = -p;
          bnd[sgn] = 1;
        } else {
          hs[sgn] = h;
          val[sgn] = 0.0;
          bnd[sgn] = 0;
        }
      }
      for (int sgn = 0; sgn < 2; ++sgn) {
        const double cf = 2.0 / ((hs[0] + hs[1]) * hs[sgn]);
        A[c] += cf;
        if (bnd[sgn]) b[c] += cf * val[sgn];
        else A[slot_of[sgn] * N + c] -= cf;
      }
    }
  }
  {
    int its = 0;
    double res = 0.0;
    status = pfo_bicgstab(nx, ny, nz, A, b, phiL, 20000, 1e-14, 0, &its, &res);
    if (lin_iters) *lin_iters = its;
    if (status) goto out;
  }
  for (long c = 0; c < N; ++c) {
    if (solvent[c]) { G[c] = 0.0; continue; }
    const long k = c / ((long)nx * ny);
    const double r[3] = {origin[0] + h * (double)(c % nx), origin[1] + h * (double)((c / nx) % ny),
                         origin[2] + h * (double)k};
    double p;
    coulomb(nq, charges, coef, r, &p, NULL);
    G[c] = p + phiL[c];
  }

  /* the interface right-hand side: every face between a membrane and a solvent node */
  memset(bif, 0, sizeof(double) * N);
  for (long c = 0; c < N; ++c) {
    const int idx[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
    for (int a = 0; a < 3; ++a) {
      if (idx[a] == n3[a] - 1) continue;
      const long nb = c + st3[a];
      if (solvent[c] == solvent[nb]) continue;
      const long cm = solvent[c] ? nb : c, cs = solvent[c] ? c : nb;
      const double nsgn = solvent[c] ? -1.0 : 1.0; /* n from the membrane node to the solvent node */
      double xi[3] = {origin[0] + h * idx[0], origin[1] + h * idx[1], origin[2] + h * idx[2]};
      xi[a] += 0.5 * h;
      double p, gr[3];
      coulomb(nq, charges, coef, xi, &p, gr);
      const double dstar = nsgn * gr[a];
      /* d phi^L / dn at the midpoint from -phi* there and phi^L at the membrane node (h/2 inside) and at
       * the next node inside (3h/2), when that one is a membrane node too */
      const long cm2 = cm - (long)nsgn * st3[a];
      const int im2 = (int)((a == 0 ? cm2 % nx : a == 1 ? (cm2 / nx) % ny : cm2 / ((long)nx * ny)));
      const int im = (int)((a == 0 ? cm % nx : a == 1 ? (cm / nx) % ny : cm / ((long)nx * ny)));
      const int inside = (nsgn > 0 ? im > 0 : im < n3[a] - 1) && (im2 >= 0) && !solvent[cm2];
      const double f0 = -p, f1 = phiL[cm];
      const double dL = inside ? (8.0 * f0 - 9.0 * f1 + phiL[cm2]) / (3.0 * h) : (f0 - f1) / (0.5 * h);
      const double J = eps_m * (dstar + dL);
      const long km = cm / ((long)nx * ny), ks = cs / ((long)nx * ny);
      if (km > 0 && km < nz - 1) bif[cm] += -eps_m * J / ((eps_m + eps_s) * h);
      if (ks > 0 && ks < nz - 1) bif[cs] += -eps_s * J / ((eps_m + eps_s) * h);
    }
  }
out:
  free(A); free(b); free(phiL);
  return status;
}

/* The lagged reading of Eq. (11): the concentrations from phi and the steric potential S_prev of the
 * previous iterate, then Gamma = 1 - sum v_i C_i and the new S = ln(Gamma / Gamma^B). */
static int lagged_fermi(int ns, const double* z, const double* v, const double* p, const double* cB, double gammaB,
                        double phi, double S_prev, double* C, double* S, double* Gamma) {
  double occ = 0.0;
  for (int i = 0; i < ns; ++i) {
    C[i] = cB[i] * exp(-z[i] * phi + p[i] * S_prev);
    occ += v[i] * C[i];
  }
  const double g = 1.0 - occ;
  if (!(g > 0.0)) return PFO_E_GAMMA;
  *Gamma = g;
  *S = log(g / gammaB);
  return PFO_OK;
}

/* Rows of the fixed nodes (the filter region) become identity rows. */
static void fix_rows(long N, const unsigned char* fixed, double* A) {
  if (!fixed) return;
  for (long c = 0; c < N; ++c)
    if (fixed[c]) {
      A[c] = 1.0;
      for (int d = 1; d < 7; ++d) A[d * N + c] = 0.0;
    }
}

static int pf_solve_impl(int nx, int ny, int nz, double h, const double* origin,
                         const double* eps, const unsigned char* solvent,
                         int nq, const double* charges, double phi_lo_V, double phi_hi_V,
                         int ns, const double* z, const double* radius_A, const double* bulk_M,
                         double eps_s, double lc, double T, const pfo_nl_opts* opts,
                         double* phi_V, double* C_M, double* S, double* Gamma, double* Psi_out,
                         double* phi_hat_out, pfo_nl_report* rep, const unsigned char* fixed,
                         const double* fixed_phi_V) {
  const long N = (long)nx * ny * nz;
  const double Tv = pfo_thermal_voltage(T), lam = pfo_lambda(T);
  pfo_nl_report R = {PFO_OK, 0, 0, 0, 0.0};
  typedef int (*lin_fn)(int, int, int, const double*, const double*, double*, int, double, int, int*,
                        double*);
  if (opts->solver < 0 || opts->solver > 2 || opts->gamma_mode < 0 || opts->gamma_mode > 1) return PFO_E_INVAL;
  const lin_fn solve_pf1 = opts->solver >= 1 ? pfo_pcg : pfo_bicgstab;
  const lin_fn solve_pf2 = opts->solver == 2 ? pfo_pcg : pfo_bicgstab;
  double v[64], pr[64], cB[64], gB;
  if (ns > 64 || nx < 2 || ny < 2 || nz < 3) return PFO_E_INVAL;
  int st = pfo_species_setup(ns, z, radius_A, bulk_M, v, pr, cB, &gB);
  if (st) return st;

  double* A = malloc(sizeof(double) * 7 * N);
  double* ffix = calloc(N, sizeof(double));
  double* b = malloc(sizeof(double) * N);
  double* phi0 = calloc(N, sizeof(double));
  double* phi = malloc(sizeof(double) * N);
  double* psi = calloc(N, sizeof(double));
  double* rho = calloc(N, sizeof(double));
  double* kap = calloc(N, sizeof(double));
  double* sig = calloc(N, sizeof(double));
  double* C = calloc((size_t)ns * N, sizeof(double));
  double* Sv = calloc(N, sizeof(double));
  double* Gv = calloc(N, sizeof(double));
  double* Gdec = NULL; /* G = phi* + phi^L of the decomposition (charge_mode 1) */
  double* Slag = opts->gamma_mode == 1 ? calloc(N, sizeof(double)) : NULL; /* lagged S (gamma_mode 1) */
  if (!A || !ffix || !b || !phi0 || !phi || !psi || !rho || !kap || !sig || !C || !Sv || !Gv ||
      (opts->gamma_mode == 1 && !Slag)) {
    st = PFO_E_INVAL;
    goto out;
  }
  if (opts->charge_mode == 1) {
    /* Eqs. 5-10: G = phi* + phi^L in Omega_m, the jump terms of Eq. 8 in place of the spread charges */
    double eps_m = -1.0;
    for (long c = 0; c < N; ++c)
      if (!solvent[c]) {
        if (eps_m < 0.0) eps_m = eps[c];
        else if (eps[c] != eps_m) { st = PFO_E_INVAL; goto out; }
      }
    Gdec = calloc(N, sizeof(double));
    if (!Gdec) { st = PFO_E_INVAL; goto out; }
    if (eps_m > 0.0) {
      st = pfo_decompose(nx, ny, nz, h, origin, solvent, nq, charges, eps_m, eps_s, lam, Gdec, ffix, NULL);
      if (st) goto out;
    }
  } else if (opts->charge_mode == 0) {
    st = pfo_spread_charges(nx, ny, nz, h, origin, nq, charges, lam, ffix);
    if (st) goto out;
  } else {
    st = PFO_E_INVAL;
    goto out;
  }
  const double lo_hat = phi_lo_V / Tv, hi_hat = phi_hi_V / Tv;
  const long plane = (long)nx * ny;
#define PFO_SET_DIRICHLET(vec)                                        \
  for (long c = 0; c < plane; ++c) { vec[c] = lo_hat; vec[N - plane + c] = hi_hat; } \
  if (fixed)                                                          \
    for (long c = 0; c < N; ++c)                                      \
      if (fixed[c]) vec[c] = fixed_phi_V[c] / Tv;

  /* initial potential: PF2 with rho' = Psi = 0, i.e. -div(eps grad phi0) = lambda rho_fix. */
  pfo_assemble_eps(nx, ny, nz, h, eps, NULL, A);
  fix_rows(N, fixed, A);
  for (long c = 0; c < N; ++c) b[c] = ffix[c];
  PFO_SET_DIRICHLET(b);
  int its = 0;
  double res = 0.0;
  st = solve_pf2(nx, ny, nz, A, b, phi0, opts->max_lin, opts->lin_tol, opts->lin_norm, &its, &res);
  R.lin_iters_first = its;
  R.lin_iters_total += its;
  if (st) goto out;

  for (int outer = 1; outer <= opts->max_outer; ++outer) {
    /* Eq. (1) at Phi0 -> rho(Phi0) and rho'(Phi0) of Eq. (11) (scaled: kappa = -lambda rho') */
    for (long c = 0; c < N; ++c) {
      rho[c] = 0.0;
      kap[c] = 0.0;
      if (!solvent[c] || (fixed && fixed[c])) continue;
      double Ci[64], s, g;
      if (Slag) {
        st = lagged_fermi(ns, z, v, pr, cB, gB, phi0[c], Slag[c], Ci, &s, &g);
        Slag[c] = s;
      } else {
        st = pfo_fermi_point(ns, z, v, pr, cB, gB, phi0[c], Ci, &s, &g, NULL);
      }
      if (st) goto out;
      for (int i = 0; i < ns; ++i) {
        rho[c] += z[i] * Ci[i];
        kap[c] += lam * z[i] * z[i] * Ci[i];
      }
    }
    /* PF1, Eq. (12) */
    pfo_assemble_pf1(nx, ny, nz, h, solvent, eps_s, lc, A);
    fix_rows(N, fixed, A); /* Psi = 0 on the filter region, the boundary of the continuum solvent (Eq. 14) */
    for (long c = 0; c < N; ++c) b[c] = solvent[c] ? -lam * rho[c] : 0.0;
    for (long c = 0; c < plane; ++c) { b[c] = 0.0; b[N - plane + c] = 0.0; }
    st = solve_pf1(nx, ny, nz, A, b, psi, opts->max_lin, opts->lin_tol, opts->lin_norm, &its, &res);
    R.lin_iters_total += its;
    if (st) goto out;
    /* PF2, Eq. (13): -eps_s Lap phi - rho' phi = -eps_s Psi - rho' phi0 in the solvent,
     * -div(eps_m grad phi) = lambda rho_fix in the membrane */
    for (long c = 0; c < N; ++c) sig[c] = solvent[c] ? kap[c] : 0.0;
    pfo_assemble_eps(nx, ny, nz, h, eps, sig, A);
    fix_rows(N, fixed, A);
    for (long c = 0; c < N; ++c)
      b[c] = (solvent[c] ? (-eps_s * psi[c] + kap[c] * phi0[c]) : 0.0) + ffix[c];
    PFO_SET_DIRICHLET(b);
    for (long c = 0; c < N; ++c) phi[c] = phi0[c]; /* warm start */
    st = solve_pf2(nx, ny, nz, A, b, phi, opts->max_lin, opts->lin_tol, opts->lin_norm, &its, &res);
    R.lin_iters_total += its;
    if (st) goto out;
    /* relaxation and stop test */
    double delta = 0.0;
    for (long c = 0; c < N; ++c) {
      phi[c] = opts->omega * phi0[c] + (1.0 - opts->omega) * phi[c];
      const double d = fabs(phi[c] - phi0[c]);
      if (d > delta) delta = d;
      phi0[c] = phi[c];
    }
    R.outer_iters = outer;
    R.delta = delta;
    if (delta <= opts->tol_outer) break;
    if (outer == opts->max_outer) st = PFO_E_NOCONV;
  }
#undef PFO_SET_DIRICHLET
  /* concentrations, steric potential and void fraction at the final potential */
  for (long c = 0; c < N; ++c) {
    if (!solvent[c] || (fixed && fixed[c])) {
      for (int i = 0; i < ns; ++i) C[(long)i * N + c] = 0.0;
      Sv[c] = 0.0;
      Gv[c] = 0.0;
      continue;
    }
    double Ci[64], s, g;
    int st2 = Slag ? lagged_fermi(ns, z, v, pr, cB, gB, phi0[c], Slag[c], Ci, &s, &g)
                   : pfo_fermi_point(ns, z, v, pr, cB, gB, phi0[c], Ci, &s, &g, NULL);
    if (st2) { st = st2; goto out; }
    for (int i = 0; i < ns; ++i) C[(long)i * N + c] = Ci[i];
    Sv[c] = s;
    Gv[c] = g;
  }
  {
    const double m = pfo_molar_to_per_A3();
    for (long c = 0; c < N; ++c) {
      const double full = phi0[c] + (Gdec ? Gdec[c] : 0.0); /* phi = phi~ + G in Omega_m (Eq. 5) */
      if (phi_V) phi_V[c] = full * Tv;
      if (phi_hat_out) phi_hat_out[c] = full;
      if (S) S[c] = Sv[c];
      if (Gamma) Gamma[c] = Gv[c];
      if (Psi_out) Psi_out[c] = psi[c];
    }
    if (C_M) for (long c = 0; c < (long)ns * N; ++c) C_M[c] = C[c] / m;
  }
out:
  R.status = st;
  if (rep) *rep = R;
  free(A); free(ffix); free(b); free(phi0); free(phi); free(psi); free(rho); free(kap);
  free(sig); free(C); free(Sv); free(Gv); free(Gdec); free(Slag);
  return st;
}

int pfo_pf_solve(int nx, int ny, int nz, double h, const double* origin,
                 const double* eps, const unsigned char* solvent,
                 int nq, const double* charges, double phi_lo_V, double phi_hi_V,
                 int ns, const double* z, const double* radius_A, const double* bulk_M,
                 double eps_s, double lc, double T, const pfo_nl_opts* opts,
                 double* phi_V, double* C_M, double* S, double* Gamma, double* Psi_out,
                 double* phi_hat_out, pfo_nl_report* rep) {
  return pf_solve_impl(nx, ny, nz, h, origin, eps, solvent, nq, charges, phi_lo_V, phi_hi_V, ns, z, radius_A,
                       bulk_M, eps_s, lc, T, opts, phi_V, C_M, S, Gamma, Psi_out, phi_hat_out, rep, NULL, NULL);
}

int pfo_pf_solve_fixed(int nx, int ny, int nz, double h, const double* origin,
                       const double* eps, const unsigned char* solvent,
                       int nq, const double* charges, double phi_lo_V, double phi_hi_V,
                       int ns, const double* z, const double* radius_A, const double* bulk_M,
                       double eps_s, double lc, double T, const pfo_nl_opts* opts,
                       const unsigned char* fixed, const double* fixed_phi_V,
                       double* phi_V, double* C_M, double* S, double* Gamma, double* Psi_out,
                       double* phi_hat_out, pfo_nl_report* rep) {
  if (!fixed || !fixed_phi_V) return PFO_E_INVAL;
  return pf_solve_impl(nx, ny, nz, h, origin, eps, solvent, nq, charges, phi_lo_V, phi_hi_V, ns, z, radius_A,
                       bulk_M, eps_s, lc, T, opts, phi_V, C_M, S, Gamma, Psi_out, phi_hat_out, rep, fixed,
                       fixed_phi_V);
}

/* ---- the atomic site model of the filter region (Eqs. 19-20) ---------------------------------- */
int pfo_site_potentials(int nsite, const double* center, const double* radius, const double* q_ion,
                        const int* occupied, double eps_b, int nq, const double* charges, double eps_p,
                        double lambda, double* phi_hat) {
  if (nsite < 1 || nq < 0 || eps_b <= 0.0 || eps_p <= 0.0) return PFO_E_INVAL;
  for (int b = 0; b < nsite; ++b) {
    if (!(radius[b] > 0.0)) return PFO_E_INVAL;
    /* the six symmetric points on the sphere of site b: +-radius along x, y and z */
    double mean = 0.0;
    for (int k = 0; k < 6; ++k) {
      double A[3] = {center[3 * b], center[3 * b + 1], center[3 * b + 2]};
      A[k / 2] += (k % 2 ? -1.0 : 1.0) * radius[b];
      double sum = 0.0;
      for (int j = 0; j < nq; ++j) {
        const double d = sqrt((charges[4 * j] - A[0]) * (charges[4 * j] - A[0]) +
                              (charges[4 * j + 1] - A[1]) * (charges[4 * j + 1] - A[1]) +
                              (charges[4 * j + 2] - A[2]) * (charges[4 * j + 2] - A[2]));
        if (!(d > 0.0)) return PFO_E_INVAL;
        sum += charges[4 * j + 3] / (eps_p * d);
      }
      for (int m = 0; m < nsite; ++m) {
        if (m == b || !occupied[m]) continue;
        const double d = sqrt((center[3 * m] - A[0]) * (center[3 * m] - A[0]) +
                              (center[3 * m + 1] - A[1]) * (center[3 * m + 1] - A[1]) +
                              (center[3 * m + 2] - A[2]) * (center[3 * m + 2] - A[2]));
        if (!(d > 0.0)) return PFO_E_INVAL;
        sum += q_ion[m] / (eps_b * d);
      }
      mean += sum / 6.0;
    }
    const double own = occupied[b] ? q_ion[b] / (eps_b * radius[b]) : 0.0;
    phi_hat[b] = lambda / (4.0 * M_PI) * (mean + own);
  }
  return PFO_OK;
}

int pfo_site_steric(int nsite, const double* ion_radius, const int* occupied, double v_sites, double gammaB,
                    double* S) {
  if (nsite < 1 || !(v_sites > 0.0) || !(gammaB > 0.0)) return PFO_E_INVAL;
  double vol = 0.0;
  for (int m = 0; m < nsite; ++m)
    if (occupied[m]) vol += 4.0 * M_PI * ion_radius[m] * ion_radius[m] * ion_radius[m] / 3.0;
  if (!(vol < v_sites)) return PFO_E_INVAL;
  *S = log((1.0 - vol / v_sites) / gammaB);
  return PFO_OK;
}
