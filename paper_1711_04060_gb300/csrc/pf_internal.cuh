// pf_internal.cuh -- types and kernel launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

constexpr int TX = 32;           // tile width in x (one warp per row)
constexpr int TY = 8;            // tile height in y
constexpr int NTHREADS = TX * TY;
constexpr int ZC = 16;           // interior planes per z-chunk of a tile
constexpr int MAXSP = 8;
constexpr int NPART = 8;         // per-block partial values reduced by the last block

// Device-resident BiCGSTAB scalars (Table 3); written only by the last block of a kernel.
struct BicgState {
  double rho;      // r~ . r of the current residual
  double alpha, omega, beta;
  double bnorm2;   // ||b||_2^2 of the system
  double rnorm2, rinf;   // ||r||_2^2, ||r||_inf of the latest residual
  double snorm2, sinf;
  double tol;      // tolerance as given
  double tol2;     // REL2: tol^2 * ||b||^2
  int norm;        // 0 REL2, 1 ABSINF
  int iter, max_iter;
  int done, status, sexit;
  unsigned int ticket;   // arrival counter of the last-block reduction
  int pad;
};

// View of one 7-point operator in right-preconditioned form.  Rows with dinv == 0 are
// identity rows (Dirichlet or membrane rows of PF1).
template <typename T>
struct OpView {
  const T* wE;    // face coefficient between (i,j,k) and (i+1,j,k), already / h^2; at i = nx-1 it
                  // holds the mirror face of (nx-2, nx-1)
  const T* wN;    // same in y
  const T* wU;    // same in z
  const T* dinv;  // 1/diag on free rows, 0 on identity rows
  const double* diag;  // FP64 diagonal (only for FP64 full-operator applies); may be null for UNI
  T wc;           // uniform face coefficient (UNI operators)
  double diagc;   // uniform diagonal (UNI operators)
  int nx, ny, nz;
};

struct Launch {
  int blocks;       // persistent grid size for stencil kernels
  int ntiles;
  cudaStream_t stream;
};

// species constants of Eq. (1) in scaled units
struct SpeciesParams {
  int ns;
  double z[MAXSP];
  double lvc[MAXSP];    // ln(v_i cB_i) (or -inf when cB_i = 0)
  double p[MAXSP];      // v_i / v0
  double lcB[MAXSP];    // ln cB_i
  double lgB;           // ln Gamma^B
  double lam;           // lambda
};

int tiles_for(int nx, int ny, int nz);

// ---- setup (a1) ----
cudaError_t launch_faces(const double* eps, int nx, int ny, int nz, double h, double* wE, double* wN,
                         double* wU, double* dsum, cudaStream_t s);
cudaError_t launch_spread(const double* charges, int nq, double ox, double oy, double oz, double h, double lam,
                          int nx, int ny, int nz, double* f, int* err, cudaStream_t s);
// diag = dsum + sig (sig may be null, masked by solvent when smask non-null); dinv = 1/diag off the
// Dirichlet planes, 0 on them; optional FP32 copies.
cudaError_t launch_eps_diag(const double* dsum, const double* sig, const uint8_t* smask, int nx, int ny, int nz,
                            double* diag, double* dinv, float* dinv32, cudaStream_t s);
cudaError_t launch_pf1_dinv(const uint8_t* solvent, int nx, int ny, int nz, double dinvc, double* dinv,
                            float* dinv32, cudaStream_t s);
cudaError_t launch_to_f32(const double* a, float* b, long n, cudaStream_t s);
cudaError_t launch_impose(double* x, const double* b, const double* dinv, long n, cudaStream_t s);

// ---- BiCGSTAB (Table 3) ----
template <typename T, bool UNI>
cudaError_t launch_init(const OpView<T>& op, const T* x, bool x_zero, const T* b, T* r, T* rt, T* p, T* v, T* t,
                        double* part, BicgState* st, const Launch& L);
template <typename T, bool UNI>
cudaError_t launch_phase_b(const OpView<T>& op, const T* r, const T* v, const T* rt, T* t, double* part,
                           BicgState* st, const Launch& L);
template <typename T, bool UNI>
cudaError_t launch_phase_ca(const OpView<T>& op, const T* r, const T* v, const T* p, const T* t, const T* rt, T* x,
                            T* r_out, T* p_out, T* v_out, double* part, BicgState* st, int prime, const Launch& L);

// FP64 residual for iterative refinement: x += d (if d), r = b - A x; writes r32 = (float) r; fills st
// (bnorm2, rnorm2, rinf) and sets st->done when the FP64 tolerance is met.
template <bool UNI>
cudaError_t launch_refine(const OpView<double>& op, double* x, const float* d, const double* b, float* r32,
                          double* part, BicgState* st, const Launch& L);
// resets a solver state with the given stop test (all scalars zero, not done)
cudaError_t launch_set_state(BicgState* st, double tol, int norm, int max_iter, cudaStream_t s);
// sum of b^2 over the Dirichlet planes into st->bnorm2 (launch before init / refine)
cudaError_t launch_plane_bb(const double* b, int nx, int ny, int nz, BicgState* st, cudaStream_t s);
Launch make_launch(int nx, int ny, int nz, cudaStream_t s);
int max_partial_blocks();

// ---- nonlinear step (Eq. 1, Eq. 11-13, Table 4) ----
// Pointwise Fermi/steric step at phi0 (solvent nodes).  Writes b1 = -lambda rho (free PF1 rows, else 0),
// sig = kappa (solvent nodes, else 0), c2 = sig*phi0 + ffix; when C/S/G are non-null also the outputs.
cudaError_t launch_fermi(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesParams& sp,
                         int nx, int ny, int nz, double* b1, double* sig, double* c2, double* C, double* S,
                         double* G, int* err, cudaStream_t s);
// b2 = -s eps_s Psi + c2 off the Dirichlet planes, Dirichlet values on them
cudaError_t launch_pf2_rhs(const double* psi, const uint8_t* solvent, const double* c2, double eps_s, double lo,
                           double hi, int nx, int ny, int nz, double* b2, cudaStream_t s);
// phi0 <- omega phi0 + (1-omega) phi, delta = max |change| (block maxima in part, last block -> *delta)
cudaError_t launch_relax(double* phi0, const double* phi, double omega, long n, double* part, unsigned int* ticket,
                         double* delta, cudaStream_t s);
cudaError_t launch_scale(const double* a, double s, double* out, long n, cudaStream_t st);
cudaError_t launch_set_dirichlet(double* x, double lo, double hi, int nx, int ny, int nz, cudaStream_t s);

}  // namespace pf
