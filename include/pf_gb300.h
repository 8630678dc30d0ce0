/*
 * pf_gb300.h -- C ABI of the GB300 (sm_103a) Poisson-Fermi solver.
 *
 * The library solves the Poisson-Fermi (PF) model of Chen, Chen and Liu, "A GPU
 * Poisson-Fermi Solver for Ion Channel Simulations": the Fermi-like concentrations and
 * steric potential of Eq. (1), the fourth-order PF equation (2) split into the two
 * second-order equations PF1 (12) and PF2 (13) of the inexact-Newton linearisation (11),
 * discretised by the 7-point finite-difference scheme of Section 3 with the simplified
 * matched-interface (SMIB) rows of Eqs. (15)-(18), and solved by the nonlinear iteration of
 * Table 4 around Jacobi-preconditioned BiCGSTAB (Table 3).  All arithmetic of the solve runs
 * in CUDA kernels on one GPU; this header is the whole interface.
 *
 * Conventions shared by every call:
 *  - Grid: nx*ny*nz nodes, uniform spacing h (Angstrom), node (i,j,k) at
 *    origin + h*(i,j,k).  Arrays are node-major with x fastest: id = i + nx*(j + ny*k)
 *    (the index order of the diagonal storage in Section 4).  N = nx*ny*nz counts the
 *    boundary nodes, as the paper's N does.
 *  - Boundary conditions (Eq. 4): Dirichlet values on the planes k = 0 and k = nz-1,
 *    zero normal flux (mirror ghost nodes) on the four x/y sides.
 *  - Scaled units: lengths in Angstrom, concentrations in Angstrom^-3 inside the solver,
 *    potential phi_hat = e*phi/(k_B T); the constants are those of Table 1.  Inputs and
 *    outputs of pf_nonlinear_solve are in volts and mol/L.
 *  - Pointers: "host" arrays are read (or written) during the call only and stay owned by
 *    the caller.  "device" arrays are device pointers of the current CUDA device, used in
 *    stream order on the grid's stream; the call returns after its work on that stream has
 *    finished.  The library owns and frees every device buffer it allocates.
 *  - Errors: every call returns a pf_status and never aborts.  pf_last_error() gives a
 *    message for the calling thread's last failing call.  Non-convergence and breakdown
 *    still write the last iterate and the report.
 *  - Threads: one grid must not be used by two threads at once; different grids may.
 */
#ifndef PF_GB300_H
#define PF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PF_OK = 0,
  PF_E_INVAL = 1,      /* bad argument (sizes, pointers, non-neutral bath, charge off grid) */
  PF_E_OOM = 2,        /* device allocation failed, or a request can never fit the budget */
  PF_E_NOCONV = 3,     /* iteration limit reached before the tolerance */
  PF_E_BREAKDOWN = 4,  /* BiCGSTAB breakdown (rho, r~.v or omega became zero) */
  PF_E_GAMMA = 5,      /* the pointwise void-fraction root of Eq. (1) was not found */
  PF_E_CUDA = 6,       /* a CUDA runtime error (message in pf_last_error) */
  PF_E_TIMEOUT = 7,    /* a bounded device wait ran out */
  PF_PENDING = 8       /* serving: the ticket has not finished yet */
} pf_status;

typedef enum { PF_FP64 = 0, PF_MIXED = 1 } pf_precision;
/* Krylov method of a linear solve.  Section 3 names the Laplace/Poisson system (Eq. 9) and PF1 (Eq. 12)
 * symmetric, PF2 (Eq. 13) not in general; with the zero-jump faces this library assembles, PF2 is symmetric in
 * the side-weighted inner product too.  PF_CG_SYMMETRIC: Jacobi-preconditioned conjugate gradients
 * (Chronopoulos-Gear form, one pass per iteration) for the Poisson and PF1 systems, BiCGSTAB for PF2;
 * PF_CG_ALL: conjugate gradients for all three. */
typedef enum { PF_BICGSTAB = 0, PF_CG_SYMMETRIC = 1, PF_CG_ALL = 2 } pf_method;

/* Linear operators that pf_linear_solve can invert (all 7-point, Section 3):
 *  PF_OP_POISSON: (A x)_c = (1/h^2) sum_nb eps_f (x_c - x_nb), eps_f = 2 eps_a eps_b/(eps_a+eps_b)
 *                 (Eqs. 7 and 15-18 with zero jump), identity rows on k = 0, nz-1;
 *  PF_OP_PF2:     the same plus s_c kappa_c x_c (Eq. 13 with kappa = -lambda rho'(phi_0)),
 *                 kappa from pf_set_kappa (zero until set), s_c = 1 at solvent nodes;
 *  PF_OP_PF1:     eps_s (lc^2/h^2 sum_nb (x_c - x_nb) + x_c) at solvent nodes off the Dirichlet
 *                 planes (Eq. 12), identity rows at membrane nodes and on k = 0, nz-1 (Eq. 14). */
typedef enum { PF_OP_POISSON = 0, PF_OP_PF1 = 1, PF_OP_PF2 = 2 } pf_operator;

typedef enum { PF_MEM_HOST = 0, PF_MEM_DEVICE = 1 } pf_mem;

/* Stop tests: PF_NORM_REL2 stops when ||b - A x||_2 <= tol * ||b||_2; PF_NORM_ABSINF stops
 * when ||b - A x||_inf < tol (the stop test of Table 3). */
typedef enum { PF_NORM_REL2 = 0, PF_NORM_ABSINF = 1 } pf_norm;

#define PF_MAX_SPECIES 8

typedef struct pf_grid pf_grid;

typedef struct {
  int z;            /* charge number (q_i = z e); water has z = 0 and comes last */
  double radius_A;  /* hard-sphere radius a_i (Angstrom), v_i = 4 pi a_i^3 / 3 */
  double bulk_M;    /* bulk concentration C_i^B (mol/L) */
} pf_species;

/* Problem data of Eqs. (1)-(4) on one grid.  All arrays are host arrays of N entries unless
 * noted; they are copied to the device by pf_set_coeffs. */
typedef struct {
  const double* eps;       /* relative dielectric at each node (eps_m in the membrane/protein,
                              eps_s in the solvent); must be > 0 */
  const uint8_t* solvent;  /* 1 = node of the solvent domain Omega_s, 0 = biomolecular domain */
  int n_charges;           /* number of fixed point charges (Eq. 3), may be 0 */
  const double* charges;   /* n_charges x 4: x, y, z (Angstrom), q (units of e); spread onto
                              the 8 corners of their cell by trilinear weights; each must lie
                              inside the grid */
  double phi_zlo_V;        /* Dirichlet potential on the plane k = 0 (volts) */
  double phi_zhi_V;        /* Dirichlet potential on the plane k = nz-1 (volts) */
  int n_species;           /* K ions + water, 1 <= n_species <= PF_MAX_SPECIES */
  const pf_species* species;
  double eps_s;            /* solvent dielectric constant of Eqs. (12)-(13) */
  double lc_A;             /* correlation length l_c (Angstrom), >= 0 */
  double T_K;              /* temperature (K); 298.15 in Table 1 */
} pf_coeffs;

typedef struct {
  int max_iter;       /* BiCGSTAB iterations (FP64) or total inner iterations (mixed) */
  double tol;         /* tolerance of the stop test named by `norm` */
  int norm;           /* pf_norm */
  int precision;      /* pf_precision: PF_FP64, or PF_MIXED = FP32 BiCGSTAB inside FP64
                         iterative refinement (true residual b - A x in FP64) */
  double inner_tol;   /* PF_MIXED: relative residual reduction of each FP32 inner solve */
  int max_refine;     /* PF_MIXED: limit on FP64 refinement steps */
  int method;         /* pf_method (PF_BICGSTAB, Table 3, by default); single-grid solves only: a batch or a
                         served request with another method is refused with PF_E_INVAL */
} pf_solve_opts;

typedef struct {
  int status;         /* pf_status of the solve */
  int iterations;     /* BiCGSTAB iterations performed (summed over inner solves) */
  int refinements;    /* PF_MIXED: FP64 residual recomputations; 0 for PF_FP64 */
  double residual;    /* final true residual: ||b-Ax||_2/||b||_2 (REL2) or ||b-Ax||_inf */
  double time_ms;     /* device time of the solve (CUDA events on the grid's stream) */
} pf_report;

typedef struct {
  double omega;       /* relaxation weight omega_PF of Tables 2 and 4 (0.3 in the paper) */
  double tol_outer;   /* stop when ||Phi - Phi_0||_inf <= tol_outer (phi_hat units), where Phi is the relaxed
                         update omega Phi_0 + (1-omega) Phi_solve of Table 4 */
  int max_outer;      /* outer (Newton) iteration limit */
  pf_solve_opts lin;  /* options of every linear solve inside the loop */
  int accel_depth;    /* 0: the paper's relaxation.  m in 1..8: Anderson acceleration of the same fixed-point
                         map with the last m differences (mixing 1 - omega); same fixed point, same stop test,
                         not in the paper.  Needs 2m + 3 more FP64 vectors on the grid. */
  double lin_forcing; /* 0: every linear solve uses lin.tol (the paper).  c > 0: the linear solves of outer
                         iteration k also stop once ||r||_2 <= eta_k ||r0||_2, r0 the residual of their warm
                         start and eta_k = min(1e-2, c * delta_{k-1}) (an inexact-Newton forcing term, not in the
                         paper; 2-norm stop only).  The outer update is then exact to a fraction eta_k of itself,
                         so the stop test on delta keeps its meaning. */
  int warm_start;     /* 0: Phi_0 from the initial PF2 solve with rho' = Psi = 0 (Table 4).  1: the iteration
                         starts from the grid's current potential: the final Phi_0 of the previous
                         pf_nonlinear_solve on this grid (so a solve stopped by max_outer resumes where it
                         stopped) or the one given to pf_set_potential; PF_E_INVAL if the grid holds none.  The
                         fixed point does not depend on the start. */
  int predict;        /* starting vector of the PF1 and PF2 solves of outer iteration k (the paper does not fix
                         it): the last solution of the same system extrapolated along its last change,
                         x_{k-1} + c (x_{k-1} - x_{k-2}).  2 (default): c = d1.d0 / d0.d0 clamped to [0, 1]
                         (d1 = x_{k-1} - x_{k-2}, d0 = x_{k-2} - x_{k-3}; in outer iteration 3, as 1).  1: c =
                         delta_{k-1} / delta_{k-2} while the outer updates shrink, else 0.  0: PF1 from the
                         previous Psi, PF2 from Phi_0.  1 and 2 hold 4 FP64 vectors, allocated on first use.
                         Either way each solve meets lin.tol; single-grid solves, batches and served requests
                         alike. */
} pf_nl_opts;

/* Output and report of pf_nonlinear_solve.  Output pointers may be NULL; `mem` says whether
 * the non-NULL ones are host or device arrays. */
typedef struct {
  double* phi_V;      /* [N] electric potential (volts) */
  double* C_M;        /* [n_species * N] concentrations (mol/L), species-major; zero outside
                         the solvent */
  double* S;          /* [N] steric potential S^trc = ln(Gamma/Gamma^B); zero outside the solvent */
  double* Gamma;      /* [N] void fraction; zero outside the solvent */
  double* Psi;        /* [N] the PF1 variable Psi of Eq. (12) (Angstrom^-2, phi_hat units) from the last
                         outer iteration */
  int mem;            /* pf_mem of the five arrays above */
  /* report */
  int status;
  int outer_iters;
  int lin_iters_total;
  int lin_iters_first;  /* iterations of the initial PF2 solve (Table 4) */
  double delta;         /* last ||Phi - Phi_0||_inf */
  double time_ms;       /* device time of the whole solve */
} pf_result;

/* Fills the options with defaults: FP64, relative 2-norm 1e-10, 20000 iterations; mixed
 * inner tolerance 0.1 (at most 1000 FP32 iterations per refinement step), 64 refinements;
 * omega 0.3, tol_outer 1e-9, 500 outer iterations, no acceleration, fixed linear tolerance. */
void pf_default_solve_opts(pf_solve_opts* o);
void pf_default_nl_opts(pf_nl_opts* o);

/* Creates a grid: nx, ny >= 2, nz >= 3, h_A > 0; origin_A[3] is the coordinate of node (0,0,0).
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream) that every later call on
 * this grid uses.  Allocates the device state of the grid (about 390 bytes per node: operators,
 * FP64 and FP32 Krylov vectors, nonlinear state and outputs); returns PF_E_OOM when that fails.
 * *out receives the handle. */
pf_status pf_create_grid(int nx, int ny, int nz, double h_A, const double origin_A[3],
                         void* cuda_stream, pf_grid** out);

/* Device bytes that pf_create_grid allocates for an nx x ny x nz grid, plus the four FP64 vectors of the
 * predicted starting vectors (pf_nl_opts.predict, allocated by the first nonlinear solve that uses them)
 * and the 2m + 3 FP64 vectors that Anderson acceleration of depth m = accel_depth adds at its first use
 * (0: none) — the figure the server's HBM budget admits requests by.  Needs no device. */
size_t pf_grid_bytes(int nx, int ny, int nz, int accel_depth);

/* Copies the problem data (host arrays) to the device and builds the operators: harmonic
 * face coefficients (Eqs. 15-18 with zero jump), diagonals and Jacobi scalings, the
 * trilinear fixed-charge source (Eq. 3) and the species constants of Eq. (1).  Validates
 * the bath (neutral, Gamma^B > 0) and the charges (inside the grid).  Resets kappa to 0. */
pf_status pf_set_coeffs(pf_grid* g, const pf_coeffs* c);

/* Sets kappa_c (Angstrom^-2) of PF_OP_PF2 from N values in host or device memory. */
pf_status pf_set_kappa(pf_grid* g, const double* kappa, int mem);

/* Sets a filter region (Section 3 with Eqs. 19-20): the nodes with fixed[c] = 1 (N bytes, 0/1) hold phi_V[c]
 * (volts; N values) as Dirichlet values of the continuum model.  Their rows become identity rows of the
 * Poisson, PF1 and PF2 operators, PF1 takes Psi = 0 there (they bound the continuum solvent, Eq. 14), and
 * pf_nonlinear_solve writes C, S and Gamma as 0 there (the site model of Eqs. 19-20 describes them).  A
 * caller computes the site potentials (Eq. 19) and maps the sites to nodes.  fixed = NULL clears the region.
 * Replacing or clearing a region rebuilds the operators, which also resets kappa.  Host or device arrays per
 * `mem`; copied.
 * pf_set_coeffs clears the region; a grid with a region cannot be solved in a batch (PF_E_INVAL) and is
 * not served. */
pf_status pf_set_filter(pf_grid* g, const uint8_t* fixed, const double* phi_V, int mem);

/* Treatment of the fixed charges.  PF_CHARGES_SPREAD (the default after pf_set_coeffs): each charge is spread
 * onto the 8 corners of its cell (Eq. 3 on the grid).  PF_CHARGES_DECOMPOSED: the potential decomposition of
 * Eqs. (5)-(10).  In the biomolecular domain phi = phi~ + G with G = phi* + phi^L, phi* the Coulomb potential of
 * the charges in the uniform membrane dielectric eps_m (Eq. 6) and phi^L the harmonic function with
 * phi^L = -phi* on the interface (the sign that keeps phi continuous; Eq. 10 prints the other) and dG/dn = 0 on
 * the x/y sides; phi~ then solves the charge-free problem whose interface rows (Eqs. 16-18) carry the jump
 * [eps dphi~/dn] = eps_m d(phi* + phi^L)/dn of Eq. (8) (again the sign of Eq. 8, not Eq. 16's) through the
 * c0 / d0 terms.  The interface sits at the midpoint of each face between a membrane and a solvent node;
 * phi^L is solved on the device with Shortley-Weller rows (Jacobi-BiCGSTAB, relative residual 1e-13).
 * pf_set_charge_mode(PF_CHARGES_DECOMPOSED) builds G and the interface right-hand side once for the current
 * coefficients; every later pf_nonlinear_solve (and batch) uses them and returns phi = phi~ + G.  Needs
 * pf_set_coeffs first, nx, ny >= 3, one dielectric value over all non-solvent nodes, every charge off the nodes
 * and every side node of the same kind as its mirror partner (PF_E_INVAL otherwise).  report (may be NULL) gets
 * the phi^L solve's iterations, residual and device time.  pf_set_coeffs returns the grid to
 * PF_CHARGES_SPREAD. */
typedef enum { PF_CHARGES_SPREAD = 0, PF_CHARGES_DECOMPOSED = 1 } pf_charge_mode;
pf_status pf_set_charge_mode(pf_grid* g, int mode, pf_report* report);

/* The decomposition's G (volts, N values; 0 in the solvent) and interface right-hand side (the scaled
 * source term that replaces the spread charges in the PF2 rows, N values) into host or device arrays per mem;
 * either may be NULL.  PF_E_INVAL unless the grid is in PF_CHARGES_DECOMPOSED mode. */
pf_status pf_get_decomposition(pf_grid* g, double* G_V, double* b_if, int mem);

/* A filter region built from the site model of Eqs. (19)-(20) on the device.  Site b is a sphere of radius
 * a_b at center_A[3b..3b+2] that may hold an ion of charge number q_ion[b] and hard-sphere radius
 * ion_radius_A[b].  Eq. (19): its scaled potential is the mean over the six points center +- a_b along x, y and z
 * of the grid's fixed charges (those of pf_set_coeffs) screened by eps_p and of the ions at the other occupied
 * sites screened by eps_b, plus its own ion q_b / (eps_b a_b) when occupied (lambda / 4 pi converts to k_BT/e).
 * The solvent nodes within max(a_b, map_radius_A) of a centre then hold that site's potential as a filter
 * region (exactly as pf_set_filter with those nodes; where spheres overlap the lowest b wins).  Eq. (20): the
 * site region's steric potential S = ln((1 - sum of the occupied ions' volumes / v_sites_A3) / Gamma^B).
 * Outputs (host, may be NULL): site_phi_V[n_sites] (volts), *site_S.  PF_E_INVAL for bad sizes or radii, a six-
 * point position on a charge or site centre, or ions that fill v_sites_A3 (nothing is changed then).
 * The choices the paper leaves open (the six points on the axes, the node mapping, V_sites as a parameter)
 * are stated here; a caller with its own mapping can use pf_set_filter with the returned potentials. */
typedef struct {
  int n_sites;
  const double* center_A;      /* n_sites x 3 (x, y, z) */
  const double* radius_A;      /* a_b > 0 */
  const double* q_ion;         /* charge number of each site's ion */
  const int* occupied;         /* 1: an ion occupies the site */
  const double* ion_radius_A;  /* hard-sphere radius of each site's ion (Eq. 20) */
  double eps_b;                /* dielectric of the site region */
  double eps_p;                /* dielectric screening the protein's fixed charges */
  double map_radius_A;         /* >= 0: nodes within max(a_b, map_radius_A) of a centre are that site's */
  double v_sites_A3;           /* volume of the site region (Eq. 20), > 0 */
} pf_sites;

pf_status pf_set_filter_sites(pf_grid* g, const pf_sites* sites, double* site_phi_V, double* site_S);

/* Sets the grid's potential Phi_0 (phi_V: N values in volts, node-major, host or device per `mem`) as the
 * start of the next pf_nonlinear_solve with warm_start = 1: a checkpoint written from pf_result.phi_V, or a
 * caller's guess.  Psi restarts from 0.  Needs pf_set_coeffs first (which forgets any potential). */
pf_status pf_set_potential(pf_grid* g, const double* phi_V, int mem);

/* Solves A x = b for the operator `op` (Table 3, Jacobi-preconditioned BiCGSTAB, preconditioner
 * applied from the right).  b and x have N entries in host or device memory (`mem`); x holds the
 * initial guess on entry and the solution on return; on identity rows x is first set to b.
 * opts may be NULL (defaults); report may be NULL. */
pf_status pf_linear_solve(pf_grid* g, int op, const double* b, double* x, int mem,
                          const pf_solve_opts* opts, pf_report* report);

/* The same solve by Jacobi-preconditioned conjugate gradients, for the systems Section 3 calls
 * symmetric (PF_OP_POISSON, the Laplace-type operator of Eq. 9, and PF_OP_PF1, Eq. 12) and for
 * PF_OP_PF2 (Eq. 13), symmetric as well with the zero-jump faces of Eqs. (15)-(18) when kappa >= 0.
 * The stored operators are symmetric in the inner product that weights a node by 1/2 for each x or
 * y side it lies on (the mirror ghosts of Eq. 4 double a side row's inward coupling); CG runs in that
 * inner product, one operator product per iteration.  Same arguments, layouts, stop tests and report
 * as pf_linear_solve (iterations = CG iterations); FP64 only (PF_E_INVAL for PF_MIXED).  Returns
 * PF_E_BREAKDOWN when a search direction has p.Ap <= 0 (an operator that is not positive definite,
 * e.g. a negative kappa), PF_E_NOCONV at max_iter; x then holds the last iterate. */
pf_status pf_linear_solve_cg(pf_grid* g, int op, const double* b, double* x, int mem,
                             const pf_solve_opts* opts, pf_report* report);

/* Runs the PF nonlinear iteration of Table 4 with the data of pf_set_coeffs: the initial PF2
 * solve with rho' = Psi = 0, then {Fermi/steric update (Eq. 1) -> PF1 solve (Eq. 12) -> PF2
 * solve (Eq. 13) -> Phi = omega Phi_0 + (1-omega) Phi, delta = ||Phi - Phi_0||_inf} until
 * delta <= tol_outer, and finally the concentrations, S and Gamma at the converged potential.
 * opts may be NULL (defaults).  The result structure receives the outputs and the report. */
pf_status pf_nonlinear_solve(pf_grid* g, const pf_nl_opts* opts, pf_result* res);

/* ---- profiling: device time per kernel kind on one grid ----------------------------------- */
enum {
  PF_PROF_INIT = 0,        /* BiCGSTAB start: r0 = b - A x0 (Table 3) */
  PF_PROF_B_FP64 = 1,      /* phase B in FP64: s, t = A M^-1 s and its inner products (omega),
                              variable-dielectric operators (PF_OP_POISSON, PF_OP_PF2) */
  PF_PROF_CA_FP64 = 2,     /* phase C+A in FP64: x, r updates, next p and v = A M^-1 p and
                              the inner products of rho and alpha, variable-dielectric operators */
  PF_PROF_B_FP32 = 3,      /* the same two phases in FP32 (mixed precision inner solves) */
  PF_PROF_CA_FP32 = 4,
  PF_PROF_B_FP64_PF1 = 5,  /* the four phase kernels on the uniform-face PF1 operator */
  PF_PROF_CA_FP64_PF1 = 6,
  PF_PROF_B_FP32_PF1 = 7,
  PF_PROF_CA_FP32_PF1 = 8,
  PF_PROF_RESIDUAL = 9,    /* FP64 true residual b - A x of iterative refinement */
  PF_PROF_FERMI = 10,      /* pointwise Fermi/steric step of Eq. (1) */
  PF_PROF_OTHER = 11,      /* setup, right-hand sides, relaxation, output conversion */
  PF_PROF_CG_DIRECTION = 12, /* conjugate gradients: direction u = r + beta u and q = A M^-1 u with <M^-1 u, q> */
  PF_PROF_CG_UPDATE = 13,  /* conjugate gradients: x and r updates with the next inner products */
  PF_PROF_CG_PASS_FP64 = 14,      /* one-pass CG iteration (PF_CG_*) in FP64, variable-dielectric operators */
  PF_PROF_CG_PASS_FP32 = 15,      /* the same in FP32 (mixed precision inner solves) */
  PF_PROF_CG_PASS_FP64_PF1 = 16,  /* one-pass CG iteration on the PF1 operator, FP64 */
  PF_PROF_CG_PASS_FP32_PF1 = 17,  /* and FP32 */
  PF_PROF_KINDS = 18
};

typedef struct {
  long long launches;                 /* kernels launched on this grid since the last reset */
  long long count[PF_PROF_KINDS];     /* launches per kind while profiling was on */
  double ms[PF_PROF_KINDS];           /* summed device time per kind (CUDA events around each launch) */
} pf_profile;

/* on != 0 resets the counters and starts timing every kernel launch with CUDA events (a small
 * overhead per launch); on = 0 stops timing.  Launch counting is always on. */
pf_status pf_profile_enable(pf_grid* g, int on);
pf_status pf_profile_get(pf_grid* g, pf_profile* out);

/* ---- the pointwise step without allocation -----------------------------------------------
 * The paper has no counterpart: this entry point exists for callers of this library that cannot
 * allocate device memory when they need the step -- an application that owns all device memory
 * through its own arena or pool, or code running where a cudaMalloc is not allowed or would stall.
 *
 * pf_fermi_noalloc computes, at n nodes and from a given potential, the same quantities as the final
 * step of pf_nonlinear_solve: at each solvent node it finds the void fraction Gamma of the Fermi-like
 * ion and water distributions and writes the concentrations C_M (mol/L, species-major, n entries per
 * species), the steric potential S = ln(Gamma/Gamma^B) and Gamma; non-solvent nodes get zeros.
 * phi_V (volts, n entries), solvent (n bytes, 1 = solvent), C_M, S and Gamma are DEVICE pointers of
 * the current device; S or Gamma may be NULL, C_M may not; species and T_K are as in pf_coeffs.
 * warm_start = 1 starts each solvent node's root search from the ln Gamma that the previous call left
 * in the scratch array at that node (useful when a caller iterates on the same n nodes, as the
 * library's own nonlinear loop does); 0 starts from the bath value.  Both give the same root to the
 * search's tolerance, and any scratch contents are safe as a start.
 *
 * It allocates nothing: its scratch (one double of ln Gamma per node and a failure flag) is a fixed
 * array of PF_FERMI_NOALLOC_MAX_NODES + 1 doubles (8 MiB) that every GPU loading the library holds
 * until the process exits.  n above PF_FERMI_NOALLOC_MAX_NODES is rejected with PF_E_INVAL.  The
 * first call on each device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current.  The work is issued on cuda_stream (NULL = legacy default stream); every call
 * then copies the failure flag to the host and synchronises that stream, so the call returns after
 * its work has finished and cannot be made while the stream is being captured.  All calls share the
 * one array: each call clears the failure flag it needs, but calls whose GPU work overlaps (different
 * streams, or threads without ordering) race on the scratch and must be serialised by the caller.
 * Returns PF_OK, PF_E_INVAL, PF_E_GAMMA (a root was not found) or PF_E_CUDA; pf_last_error() has
 * the message. */
#define PF_FERMI_NOALLOC_MAX_NODES (1L << 20)
pf_status pf_fermi_noalloc(long n, const double* phi_V, const uint8_t* solvent, int n_species,
                           const pf_species* species, double T_K, int warm_start, double* C_M, double* S,
                           double* Gamma, void* cuda_stream);

/* Frees the grid and all its device memory.  NULL is accepted. */
pf_status pf_destroy_grid(pf_grid* g);

/* Self-test of failure detection without a fault: a one-block kernel waits, with the bounded wait that
 * guards every TMA stage of the stencil kernels, on an mbarrier on which nothing ever arrives.  Returns
 * PF_E_TIMEOUT once the wait gave up after limit_cycles clock cycles (the expected outcome; the context
 * stays usable), PF_OK if the wait completed, PF_E_CUDA on a CUDA error.  Not in the paper. */
pf_status pf_selftest_wait_timeout(unsigned long long limit_cycles, void* cuda_stream);

/* Message of the calling thread's last failing call ("" if none). */
const char* pf_last_error(void);

/* ---- batched solves: many independent problems in shared launches -------------------
 * A batch solves the problems already set on `count` grids (pf_create_grid + pf_set_coeffs,
 * any sizes) together: the nonlinear iteration of Table 4 runs for every grid in lockstep
 * (each grid stops on its own test), and each BiCGSTAB phase (Table 3) and each FP64 residual
 * of all grids still iterating is ONE launch of a batched stencil kernel in which every grid
 * owns nblk = ceil(tiles / tiles_per_block) blocks; the chunks of BiCGSTAB iterations between
 * host checks are replayed as a captured CUDA graph.  A grid's arithmetic and reduction order
 * depend only on its own size and the tiling (tiles_per_block, tile depth), so a problem's result
 * is bitwise the same in any batch with the same tiling; against pf_nonlinear_solve (another block
 * count) it agrees to the solver tolerance.  Not in the paper.
 *
 * The batch borrows the grids (they must outlive it and must not be used by another call while
 * a batch call runs); its work is queued on cuda_stream, ordered after the work queued on each
 * grid's stream before the call, and the grids' streams wait for it afterwards. */
typedef struct pf_batch pf_batch;

#define PF_BATCH_TUNE_MAX 16
/* Autotuner record: the candidate tilings (tiles per block, z-planes per 32 x 8 tile) and the device time
 * (ms) of one timed prime + 4 BiCGSTAB iterations of the batch's FP32 Poisson operators for each;
 * chosen / chosen_z = the tiling in use. */
typedef struct {
  int n;
  int tiles_per_block[PF_BATCH_TUNE_MAX];
  int z_planes[PF_BATCH_TUNE_MAX];
  float ms[PF_BATCH_TUNE_MAX];
  int chosen, chosen_z;
} pf_batch_tune;

/* PF_E_INVAL for count < 1, a NULL or repeated grid; PF_E_OOM if the launch tables cannot be allocated. */
pf_status pf_batch_create(pf_grid* const* grids, int count, void* cuda_stream, pf_batch** out);

/* tiles_per_block >= 1 pins the block split (reproducible results across runs) with the current tile depth
 * (32 z-planes unless tuned or set); 0 makes the next solve run the autotuner first (the default). */
pf_status pf_batch_set_tiles_per_block(pf_batch* b, int tiles_per_block);

/* Pins both: tiles per block (>= 1) and the tile depth in z (4..256 interior planes per 32 x 8 tile). */
pf_status pf_batch_set_tiling(pf_batch* b, int tiles_per_block, int z_planes);

/* Runs the autotuner now (needs the coefficients on every grid); *out (may be NULL) gets its record.
 * It uses the grids' FP32 scratch vectors, which every solve re-initialises. */
pf_status pf_batch_autotune(pf_batch* b, pf_batch_tune* out);
pf_status pf_batch_get_tune(pf_batch* b, pf_batch_tune* out);

/* pf_nonlinear_solve for every grid of the batch with the same options; results[i] (count entries)
 * receives grid i's outputs and report, results[i].time_ms the whole batch's device time.  Returns
 * PF_OK when every problem converged, else the first failing status (each results[i].status holds
 * its own).  accel_depth and lin_forcing work per grid as in pf_nonlinear_solve. */
pf_status pf_batch_nonlinear_solve(pf_batch* b, const pf_nl_opts* opts, pf_result* results);

/* Where the time of the last pf_batch_nonlinear_solve went: the engine's ticks (one step of every problem's
 * state machine, its shared launches and the read-back of all problems' solver states), their summed host wall
 * time, and the summed device span of each tick's work (from its first launch to the state read-back, CUDA
 * events on the batch stream).  wall_ms - device_ms is the host's share between ticks; device_ms / wall_ms
 * the fraction of the ticks' time the device had work queued.  Not in the paper. */
typedef struct {
  long long ticks;
  double wall_ms;
  double device_ms;
} pf_batch_stats;
pf_status pf_batch_get_stats(pf_batch* b, pf_batch_stats* out);

/* Frees the batch (not its grids). */
pf_status pf_batch_destroy(pf_batch* b);

/* ---- serving: continuous batching of PF solves -------------------------------------
 * A server runs one scheduler thread over a batched engine (the machinery of pf_batch with 4
 * tiles per block).  Between two engine steps it admits queued requests, first fit in arrival
 * order, while fewer than max_slots are in flight and the request's device state fits the
 * remaining HBM budget; every step runs one outer iteration of all requests in flight in shared
 * batched launches, so a request that arrives while others run joins their launches at the next
 * step.  Each request's state stays on the device until it finishes; then its outputs go to host
 * memory and its device memory returns to the budget at once.  A request's result is bitwise that
 * of pf_batch_nonlinear_solve on a batch of this problem alone with tiles_per_block 4, and agrees
 * with pf_nonlinear_solve to the solver tolerance. */
typedef struct pf_server pf_server;

typedef struct {
  int nx, ny, nz;
  double h_A;
  double origin_A[3];
  pf_coeffs coeffs;   /* host arrays; copied by pf_submit, the caller may free them afterwards */
  pf_nl_opts opts;
  const double* phi0_V; /* optional host array (N values, volts; copied): the solve starts from this potential
                           (warm start, as pf_set_potential + warm_start = 1); NULL: the paper's start */
} pf_request;

/* hbm_budget_bytes: device memory the server may hold for problem state; max_slots: problems
 * in flight at once (>= 1). */
pf_status pf_server_create(size_t hbm_budget_bytes, int max_slots, pf_server** out);

/* Queues a request and returns at once with a ticket.  PF_E_OOM if the request alone needs
 * more than the whole budget (it could never be admitted); PF_E_INVAL for bad data. */
pf_status pf_submit(pf_server* s, const pf_request* req, uint64_t* ticket);

/* *done = 1 when the ticket has finished: the outputs (host arrays in `res`, `res->mem` must be
 * PF_MEM_HOST) and the report are written and the ticket is released; returns the solve's
 * status.  *done = 0 and PF_PENDING while it is queued or running.  With res == NULL the call
 * only reports *done (PF_OK when finished) and keeps the result for a later poll. */
pf_status pf_poll(pf_server* s, uint64_t ticket, pf_result* res, int* done);

/* Stops the scheduler, cancels queued requests and frees everything. */
pf_status pf_server_destroy(pf_server* s);

#ifdef __cplusplus
}
#endif
#endif
