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

}  // namespace pf
