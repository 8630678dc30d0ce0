// pf_filter.cu -- the filter region of Eqs. (19)-(20) coupled to the continuum model (Section 3): its nodes
// hold the site potentials as Dirichlet values, so their rows become identity rows (a zero Jacobi scaling,
// the mark the solver kernels already use for fixed nodes), their right-hand sides carry the values, PF1
// takes Psi = 0 there (they bound the continuum solvent, Eq. 14) and they hold no continuum
// concentrations.  Elementwise kernels over the padded layout, launched only when a filter is set.
#include "pf_filter.cuh"

namespace pf {
namespace {

constexpr int FT = 256;

// one block per (j, k) row, threads over i
#define PF_FILTER_ROWS(g)                                                   \
  for (long row = blockIdx.x; row < (long)(g).ny * (g).nz; row += gridDim.x) \
    for (int i = threadIdx.x; i < (g).nx; i += blockDim.x)

int blocks_for(const Geom& g) {
  const long rows = (long)g.ny * g.nz;
  return (int)(rows < 65535 ? (rows > 0 ? rows : 1) : 65535);
}

__global__ void k_filter_rows(const uint8_t* __restrict__ fixed, Geom g, double* dinv, double* diag, float* dinv32) {
  PF_FILTER_ROWS(g) {
    const long c = i + g.px * row;
    if (!fixed[c]) continue;
    dinv[c] = 0.0;
    if (diag) diag[c] = 1.0;
    if (dinv32) dinv32[c] = 0.0f;
  }
}

__global__ void k_filter_values(const uint8_t* __restrict__ fixed, const double* __restrict__ value, Geom g,
                                double* b) {
  PF_FILTER_ROWS(g) {
    const long c = i + g.px * row;
    if (fixed[c]) b[c] = value[c];
  }
}

__global__ void k_filter_zero(const uint8_t* __restrict__ fixed, Geom g, double* a, int count) {
  PF_FILTER_ROWS(g) {
    const long c = i + g.px * row;
    if (!fixed[c]) continue;
    for (int f = 0; f < count; ++f) a[(long)f * g.np + c] = 0.0;
  }
}

}  // namespace

cudaError_t launch_filter_rows(const uint8_t* fixed, const Geom& g, double* dinv, double* diag, float* dinv32,
                               cudaStream_t s) {
  k_filter_rows<<<blocks_for(g), FT, 0, s>>>(fixed, g, dinv, diag, dinv32);
  return cudaGetLastError();
}

cudaError_t launch_filter_values(const uint8_t* fixed, const double* value, const Geom& g, double* b,
                                 cudaStream_t s) {
  k_filter_values<<<blocks_for(g), FT, 0, s>>>(fixed, value, g, b);
  return cudaGetLastError();
}

cudaError_t launch_filter_zero(const uint8_t* fixed, const Geom& g, double* a, int count, cudaStream_t s) {
  k_filter_zero<<<blocks_for(g), FT, 0, s>>>(fixed, g, a, count);
  return cudaGetLastError();
}

}  // namespace pf
