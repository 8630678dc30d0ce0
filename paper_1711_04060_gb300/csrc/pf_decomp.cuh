// pf_decomp.cuh -- launchers of the potential-decomposition kernels (pf_decomp.cu): the Coulomb potential of
// the fixed charges (Eq. 6), the harmonic correction phi^L (Eqs. 9-10) and the interface right-hand side of
// the jump (Eq. 8 through the SMIB rows 16-18) that replaces the spread charges.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Inputs shared by the decomposition kernels.  Arrays use the grid's padded layout.
struct DecompArgs {
  const double* ch;          // charges x, y, z (A), q (e); nq of them
  int nq;
  double coef;               // lambda / (4 pi eps_m): phi* in units of k_BT/e
  double ox, oy, oz, h;      // node (i, j, k) at origin + h (i, j, k)
  double eps_m, eps_s;
  const uint8_t* solvent;
  Geom g;
  int* err;                  // 1: a charge within 1e-6 h of a node; 2: a side node unlike its mirror partner
};

// The phi^L system as a 7-diagonal matrix (Section 4 order: A0 diagonal, then east, west, south, north, down, up)
// with its right-hand side: -Lap_h phi^L = 0 at membrane nodes off the Dirichlet planes, Shortley-Weller
// differences to the interface midpoints (distance h/2, value -phi*), dG/dn = 0 on the x/y sides; identity rows
// at solvent nodes (value 0) and on the planes (value -phi*, so that G = 0 there).
cudaError_t launch_phiL_rows(const DecompArgs& a, double* const A[7], double* b, cudaStream_t s);
// Right-preconditioned Jacobi BiCGSTAB (Table 3 with M = diag A) on that matrix, device-side scalars: start
// (x = b on identity rows, r = r~ = b - A x, p = v = 0), then [direction, s/t, update] launches per iteration.
struct DiaState {
  double rho, alpha, omega, beta, bnorm2, rnorm2, tol2;
  int iter, max_iter, done, status, sexit;
  unsigned int ticket;
};
struct DiaVecs {
  double *x, *b, *r, *rt, *p[2], *v[2], *t;
};
cudaError_t launch_dia_start(const double* const A[7], const DiaVecs& w, const Geom& g, double tol, int max_iter,
                             double* part, DiaState* st, cudaStream_t s);
cudaError_t launch_dia_iteration(const double* const A[7], const DiaVecs& w, int cur, const Geom& g, double* part,
                                 DiaState* st, cudaStream_t s);
// G = phi* + phi^L at membrane nodes, 0 in the solvent.
cudaError_t launch_decomp_G(const DecompArgs& a, const double* phiL, double* G, cudaStream_t s);
// The interface right-hand side: for each face between a membrane node and a solvent node, the jump
// J = eps_m (d phi*/dn + d phi^L/dn) at the face midpoint (n from the membrane to the solvent), added to the
// membrane node's row as -eps_m J / ((eps_m + eps_s) h) and to the solvent node's as -eps_s J / ((eps_m + eps_s) h)
// on the interior planes; d phi^L/dn from the one-sided quadratic through the midpoint and two membrane nodes
// (one node when the second is not a membrane node).
cudaError_t launch_decomp_bif(const DecompArgs& a, const double* phiL, double* bif, cudaStream_t s);
// out = (phi + G) * scale (G may be null: out = phi * scale)
cudaError_t launch_add_scale(const double* phi, const double* G, double scale, double* out, long n, cudaStream_t s);

}  // namespace pf
