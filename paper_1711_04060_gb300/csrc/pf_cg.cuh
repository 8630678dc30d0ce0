// pf_cg.cuh -- launchers of the conjugate-gradient kernels (pf_cg.cu) for the symmetric systems of
// Section 3, FP64.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// The operator as the BiCGSTAB kernels see it: Jacobi scalings (0 on identity rows), the diagonal
// (diag, or the constant diagc when diag is null) and the east/north/up faces (or the constant wc).
struct CgOperator {
  const double* dinv;
  const double* diag;
  const double *wE, *wN, *wU;
  double wc, diagc;
};

// r = b - A x, u = 0 (u may be null), and the state's norms, rho = <r, M^-1 r>_w and stop test
cudaError_t launch_cg_start(const CgOperator& a, const Geom& g, const double* b, const double* x, double* r,
                            double* u, double* part, BicgState* st, cudaStream_t s);
// un = r + beta uo, q = A M^-1 un, alpha
cudaError_t launch_cg_direction(const CgOperator& a, const Geom& g, const double* r, const double* uo, double* un,
                                double* q, double* part, BicgState* st, cudaStream_t s);
// x += alpha M^-1 un, r -= alpha q, stop test, beta
cudaError_t launch_cg_update(const CgOperator& a, const Geom& g, const double* un, const double* q, double* x,
                             double* r, double* part, BicgState* st, cudaStream_t s);

}  // namespace pf
