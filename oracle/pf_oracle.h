/*
 * pf_oracle.h -- plain, slow FP64 CPU oracle of the Poisson-Fermi (PF) solver of
 * "A GPU Poisson-Fermi Solver for Ion Channel Simulations" (Chen, Chen, Liu).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code; only the tests, the package's smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; its status codes are restated here with the same numbers so that
 * reports can be compared.
 *
 * Units used throughout (scaled form of Eqs. (1)-(3), (11)-(13)):
 *   lengths in Angstrom, concentrations in Angstrom^-3, potential phi_hat = e*phi/(k_B T),
 *   lambda = e^2 / (eps0 * k_B * T * 1 Angstrom) with the constants of Table 1.
 * Node index id = i + nx*(j + ny*k), x fastest, as the DIA storage of Section 4 orders it.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PFO_OK = 0,
  PFO_E_INVAL = 1,
  PFO_E_NOCONV = 3,
  PFO_E_BREAKDOWN = 4,
  PFO_E_GAMMA = 5
};

/* ---- constants (Table 1) ------------------------------------------------ */
double pfo_thermal_voltage(double T);   /* k_B T / e in volts */
double pfo_lambda(double T);            /* e^2/(eps0 k_B T 1A), dimensionless*A */
double pfo_molar_to_per_A3(void);       /* 1 mol/L in Angstrom^-3 (N_A * 1e-27) */

/* ---- species (Eq. 1 definitions) ---------------------------------------- */
/* From charge numbers z[i], radii a[i] (A) and bulk concentrations (mol/L) of the
 * K ions and water (the last entry, z = 0), compute v[i] = 4 pi a^3/3, p[i] = v[i]/v0
 * (v0 = mean volume over all K+1 species), cB[i] in A^-3 and Gamma^B.
 * Returns PFO_E_INVAL when the bath is not neutral or Gamma^B <= 0. */
int pfo_species_setup(int ns, const double* z, const double* radius_A, const double* bulk_M,
                      double* v, double* p, double* cB, double* gammaB);

/* ---- pointwise Fermi / steric step (Eq. 1 with Gamma from its definition) --
 * Solves Gamma + sum_i v_i cB_i exp(-z_i phi) (Gamma/GammaB)^{p_i} = 1 for Gamma in (0,1)
 * (safeguarded Newton on u = ln Gamma), then S = ln(Gamma/GammaB),
 * C_i = cB_i exp(-z_i phi + p_i S).  Returns PFO_E_GAMMA if the root is not found. */
int pfo_fermi_point(int ns, const double* z, const double* v, const double* p, const double* cB,
                    double gammaB, double phi_hat, double* C, double* S, double* Gamma, int* iters);

/* Eq. (1) at n nodes (phi_hat[n]): C[ns * n] (species-major, A^-3), S[n], Gamma[n]; PFO_OK, or the largest
 * status of a node that failed. */
int pfo_fermi_nodes(int ns, const double* z, const double* v, const double* p, const double* cB, double gammaB,
                    long n, const double* phi_hat, double* C, double* S, double* Gamma);

/* ---- matrices in the 7-diagonal format of Section 4 ----------------------
 * A is 7*N doubles: A[0*N+i] diagonal, A[1*N+i] east (i+1), A[2*N+i] west (i-1),
 * A[3*N+i] south (i-nx), A[4*N+i] north (i+nx), A[5*N+i] down (i-nx*ny), A[6*N+i] up. */

/* Variable-dielectric operator of Eqs. (7), (13), (15)-(18) with zero jump:
 * (1/h^2) sum_nb eps_f (x_c - x_nb) + sigma_c x_c at nodes 0<k<nz-1, identity rows on the
 * planes k=0 and k=nz-1 (Dirichlet, Eq. 4), mirror ghosts on the x/y sides (zero flux, Eq. 4).
 * eps_f is the harmonic mean 2 eps_a eps_b/(eps_a+eps_b).  sigma may be NULL (zero). */
int pfo_assemble_eps(int nx, int ny, int nz, double h, const double* eps, const double* sigma,
                     double* A);

/* PF1 operator of Eqs. (12), (14): eps_s*(lc^2 (-Lap_h) + 1) at solvent nodes off the
 * Dirichlet planes; identity rows (Psi = 0) at membrane nodes and on the planes k=0, nz-1;
 * mirror ghosts on the x/y sides. */
int pfo_assemble_pf1(int nx, int ny, int nz, double h, const unsigned char* solvent,
                     double eps_s, double lc, double* A);

void pfo_dia_apply(int nx, int ny, int nz, const double* A, const double* x, double* y);

/* Right-preconditioned Jacobi BiCGSTAB (van der Vorst; the preconditioned form of the
 * Templates book), Table 3.  Before iterating, x is set to b on identity rows.
 * norm_mode 0: stop when ||r||_2 <= tol*||b||_2;  norm_mode 1: stop when ||r||_inf < tol
 * (the test of Table 3).  max_it iterations at most.  Returns PFO_OK, PFO_E_NOCONV or
 * PFO_E_BREAKDOWN; *iters and *res (the final residual measure of the chosen norm,
 * relative for mode 0) are always written. */
int pfo_bicgstab(int nx, int ny, int nz, const double* A, const double* b, double* x,
                 int max_it, double tol, int norm_mode, int* iters, double* res);

/* Jacobi-preconditioned conjugate gradients for the symmetric systems of Section 3 (the Laplace
 * equation (9) and PF1 (12)), in the inner product weighted by 1/2 per mirrored side direction
 * under which the operators of pfo_assemble_eps / pfo_assemble_pf1 are self-adjoint (see
 * pfo_weighted_asymmetry).  Same arguments, stop tests and results as pfo_bicgstab; returns
 * PFO_E_INVAL when diag(A) is not positive or A is not symmetric in that inner product, and
 * PFO_E_BREAKDOWN when a search direction has p.Ap <= 0 (A not positive definite). */
int pfo_pcg(int nx, int ny, int nz, const double* A, const double* b, double* x,
            int max_it, double tol, int norm_mode, int* iters, double* res);

/* max |w_c A_cn - w_n A_nc| / max |w_c A_cn| over neighbouring rows that are not identity rows,
 * with w = 1/2 per x or y side the node lies on. */
double pfo_weighted_asymmetry(int nx, int ny, int nz, const double* A);

/* Trilinear spreading of point charges q_j (units of e) at (x,y,z) in A onto the grid
 * nodes: adds lambda*q_j*w/h^3 to f at the 8 corners of the cell holding the charge. */
int pfo_spread_charges(int nx, int ny, int nz, double h, const double* origin, int nq,
                       const double* charges, double lambda, double* f);

/* ---- potential decomposition (Eqs. 5-10) and interface right-hand side (Eqs. 8, 16-18) ----
 * For point charges (x, y, z in A, q in e) strictly inside Omega_m (the non-solvent nodes, dielectric
 * eps_m; solvent eps_s), writes G = phi* + phi^L at the membrane nodes (0 at solvent nodes; phi* the
 * Coulomb potential lambda q / (4 pi eps_m r), phi^L harmonic in Omega_m with G = 0 on the interface and
 * zero normal derivative of G on the x/y sides) and bif, the SMIB jump terms c0/h^2, d0/h^2 on the
 * membrane and solvent rows next to each interface face (midpoint interface).  The potential is then
 * phi~ + G in Omega_m and phi~ in Omega_s, where phi~ solves the harmonic-face operator with bif added
 * to its right-hand side and no spread charges.  PFO_E_INVAL when a charge lies outside the box or on a
 * node, or when a side node and its mirror partner differ in kind.  lin_iters (may be NULL) receives
 * the BiCGSTAB iterations of the phi^L solve. */
int pfo_decompose(int nx, int ny, int nz, double h, const double* origin, const unsigned char* solvent,
                  int nq, const double* charges, double eps_m, double eps_s, double lambda, double* G,
                  double* bif, int* lin_iters);

/* ---- nonlinear PF solve (Table 2; the GPU variant of Table 4 computes the same) ---- */
typedef struct {
  double omega;      /* relaxation weight omega_PF of Table 2 */
  double tol_outer;  /* stop when ||Phi - Phi0||_inf <= tol_outer (phi_hat units) */
  double lin_tol;    /* linear-solver tolerance */
  int lin_norm;      /* 0: relative 2-norm, 1: absolute inf-norm */
  int max_outer;
  int max_lin;
  int solver;        /* 0: BiCGSTAB (Table 3) for every linear system; 1: conjugate gradients
                        (pfo_pcg) for PF1; 2: conjugate gradients for PF1 and PF2 (symmetric in the
                        zero-jump reading of Eqs. 15-18) */
  int charge_mode;   /* 0: fixed charges spread trilinearly onto the grid (Eq. 3 on the grid); 1: the
                        potential decomposition of Eqs. 5-10 (pfo_decompose): the interface right-hand
                        side replaces the spread charges and phi = phi~ + G is returned in Omega_m.  Mode 1
                        needs one dielectric value on all non-solvent nodes and charges inside Omega_m. */
  int gamma_mode;    /* 0: Gamma of Eq. (1) as the root of its own definition at every node (default);
                        1: the lagged reading of Eq. (11): C_i = cB_i exp(-z_i phi + p_i S) with S from the
                        previous outer iterate (0 at the start), then Gamma = 1 - sum v_i C_i and
                        S = ln(Gamma / Gamma^B); PFO_E_GAMMA when Gamma <= 0.  Same fixed point. */
} pfo_nl_opts;

typedef struct {
  int status;
  int outer_iters;
  int lin_iters_total;
  int lin_iters_first;   /* iterations of the initial PF2 solve (Table 2) */
  double delta;          /* last ||Phi - Phi0||_inf */
} pfo_nl_report;

/* Inputs: eps[N] relative dielectric, solvent[N] (1 = solvent node), nq charges (x,y,z,q),
 * Dirichlet potentials (volts) at k=0 and k=nz-1, ns species (z, radius A, bulk mol/L; water
 * last), eps_s (solvent dielectric of Eqs. 12-13), lc (A), T (K).
 * Outputs (any may be NULL): phi_V[N] (volts), C_M[ns*N] (mol/L, species-major), S[N],
 * Gamma[N], Psi[N] (PF1 variable), phi_hat[N]. */
int pfo_pf_solve(int nx, int ny, int nz, double h, const double* origin,
                 const double* eps, const unsigned char* solvent,
                 int nq, const double* charges, double phi_lo_V, double phi_hi_V,
                 int ns, const double* z, const double* radius_A, const double* bulk_M,
                 double eps_s, double lc, double T, const pfo_nl_opts* opts,
                 double* phi_V, double* C_M, double* S, double* Gamma, double* Psi,
                 double* phi_hat_out, pfo_nl_report* rep);

/* The same solve with a filter region (Section 3, Eqs. 19-20 coupling): nodes with fixed[c] != 0 hold the
 * potential fixed_phi_V[c] (volts) as a Dirichlet value of PF2 and of the initial solve, PF1 takes Psi = 0
 * there (they bound the continuum solvent, Eq. 14), and they carry no continuum concentrations (C, S,
 * Gamma written as 0). */
int pfo_pf_solve_fixed(int nx, int ny, int nz, double h, const double* origin,
                       const double* eps, const unsigned char* solvent,
                       int nq, const double* charges, double phi_lo_V, double phi_hi_V,
                       int ns, const double* z, const double* radius_A, const double* bulk_M,
                       double eps_s, double lc, double T, const pfo_nl_opts* opts,
                       const unsigned char* fixed, const double* fixed_phi_V,
                       double* phi_V, double* C_M, double* S, double* Gamma, double* Psi_out,
                       double* phi_hat_out, pfo_nl_report* rep);

/* Eq. (19): the scaled potential phi_hat_b = e phi_b / k_B T of each of nsite spherical sites (centres x, y, z
 * in A, radii in A), the mean over the six points +-radius along x, y, z of the protein charges (x, y, z, q)
 * screened by eps_p and of the ions q_ion[m] at the other occupied sites screened by eps_b, plus the site's
 * own ion q_ion[b] / (eps_b radius[b]) when occupied; lambda/(4 pi) converts to scaled units. */
int pfo_site_potentials(int nsite, const double* center, const double* radius, const double* q_ion,
                        const int* occupied, double eps_b, int nq, const double* charges, double eps_p,
                        double lambda, double* phi_hat);

/* Eq. (20): S = ln((1 - sum_m v_m / V_sites) / Gamma^B), v_m = 4 pi a_m^3 / 3 of the ion at each occupied
 * site; V_sites (A^3) is the volume of the site region, a parameter (the paper does not give it).
 * PFO_E_INVAL when the ions fill V_sites. */
int pfo_site_steric(int nsite, const double* ion_radius, const int* occupied, double v_sites, double gammaB,
                    double* S);

#ifdef __cplusplus
}
#endif
#endif
