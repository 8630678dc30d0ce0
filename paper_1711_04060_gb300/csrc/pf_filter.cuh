// pf_filter.cuh -- launchers of the filter-region kernels (pf_filter.cu): nodes of the filter region of
// Eqs. (19)-(20) held at given potentials as Dirichlet values of the continuum solves.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// At every fixed node: dinv = 0 (an identity row, which the solver kernels honour), diag = 1 when diag is
// given, dinv32 = 0 when given.
cudaError_t launch_filter_rows(const uint8_t* fixed, const Geom& g, double* dinv, double* diag, float* dinv32,
                               cudaStream_t s);
// b = value at every fixed node
cudaError_t launch_filter_values(const uint8_t* fixed, const double* value, const Geom& g, double* b,
                                 cudaStream_t s);
// count consecutive padded fields of a (stride g.np) set to 0 at every fixed node
cudaError_t launch_filter_zero(const uint8_t* fixed, const Geom& g, double* a, int count, cudaStream_t s);

// Site model of the filter region.  site = n x 8 doubles per site: centre x, y, z (A), radius a_b (A), ion
// charge number q_b, occupied (0/1), ion radius (A), unused.  Eq. (19): phi_hat[b] = lambda/(4 pi) times
// the mean over the six points centre +- a_b along x, y, z of sum_j q_j / (eps_p d) over the charges
// (x, y, z, q; nq of them) and sum_m q_m / (eps_b d) over the other occupied sites, plus q_b / (eps_b a_b)
// when site b is occupied; err = 1 when a point coincides with a charge or a site centre.  Eq. (20): *S =
// ln((1 - sum over occupied sites of 4 pi r^3 / 3) / V_sites) / Gamma^B), err = 2 when the ions fill V_sites.
cudaError_t launch_site_potentials(const double* site, int n, const double* charges, int nq, double eps_b,
                                   double eps_p, double lam, double v_sites, double lgB, double* phi_hat, double* S,
                                   int* err, cudaStream_t s);
// fixed[c] = 1 and value[c] = phi_hat[b] at every solvent node within max(a_b, map_r) of site b's centre (the
// lowest b when spheres overlap); other nodes fixed[c] = 0.  Node (i, j, k) sits at origin + h (i, j, k).
cudaError_t launch_site_map(const double* site, int n, const double* phi_hat, const uint8_t* solvent, const Geom& g,
                            double ox, double oy, double oz, double h, double map_r, uint8_t* fixed, double* value,
                            cudaStream_t s);

}  // namespace pf
