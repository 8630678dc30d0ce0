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

constexpr int SITE_T = 256;

__device__ __forceinline__ double dist3(double ax, double ay, double az, double bx, double by, double bz) {
  return sqrt((ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz));
}

// One block per site: threads take (point, source) pairs of the six points of Eq. (19) against the charges and
// the other occupied sites; a fixed-order block reduction gives the mean.  Block 0's thread 0 also evaluates
// Eq. (20).
__global__ void __launch_bounds__(SITE_T) k_site_potentials(const double* __restrict__ site, int n,
                                                            const double* __restrict__ ch, int nq, double eps_b,
                                                            double eps_p, double lam, double v_sites, double lgB,
                                                            double* phi_hat, double* S, int* err) {
  __shared__ double red[SITE_T];
  const int b = blockIdx.x;
  const double* sb = site + 8 * b;
  const int per_point = nq + n;
  double acc = 0.0;
  for (int w = threadIdx.x; w < 6 * per_point; w += SITE_T) {
    const int k = w / per_point, src = w - k * per_point;
    double A[3] = {sb[0], sb[1], sb[2]};
    A[k / 2] += (k % 2 ? -1.0 : 1.0) * sb[3];
    if (src < nq) {
      const double d = dist3(ch[4 * src], ch[4 * src + 1], ch[4 * src + 2], A[0], A[1], A[2]);
      if (!(d > 0.0)) atomicExch(err, 1);
      else acc += ch[4 * src + 3] / (eps_p * d);
    } else {
      const int m = src - nq;
      const double* sm = site + 8 * m;
      if (m == b || sm[5] == 0.0) continue;
      const double d = dist3(sm[0], sm[1], sm[2], A[0], A[1], A[2]);
      if (!(d > 0.0)) atomicExch(err, 1);
      else acc += sm[4] / (eps_b * d);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = SITE_T / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double own = sb[5] != 0.0 ? sb[4] / (eps_b * sb[3]) : 0.0;
    phi_hat[b] = lam / (4.0 * M_PI) * (red[0] / 6.0 + own);
    if (b == 0 && S) {
      double vol = 0.0;
      for (int m = 0; m < n; ++m)
        if (site[8 * m + 5] != 0.0) vol += 4.0 * M_PI * site[8 * m + 6] * site[8 * m + 6] * site[8 * m + 6] / 3.0;
      if (!(vol < v_sites)) atomicExch(err, 2);
      else *S = log(1.0 - vol / v_sites) - lgB;
    }
  }
}

__global__ void k_site_map(const double* __restrict__ site, int n, const double* __restrict__ phi_hat,
                           const uint8_t* __restrict__ solvent, Geom g, double ox, double oy, double oz, double h,
                           double map_r, uint8_t* fixed, double* value) {
  PF_FILTER_ROWS(g) {
    const long c = i + g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const double x = ox + h * i, y = oy + h * j, z = oz + h * k;
    uint8_t f = 0;
    double v = 0.0;
    if (solvent[c]) {
      for (int b = 0; b < n; ++b) {
        const double* sb = site + 8 * b;
        const double r = fmax(sb[3], map_r);
        if (dist3(x, y, z, sb[0], sb[1], sb[2]) <= r) {
          f = 1;
          v = phi_hat[b];
          break;
        }
      }
    }
    fixed[c] = f;
    value[c] = v;
  }
}

}  // namespace

cudaError_t launch_site_potentials(const double* site, int n, const double* charges, int nq, double eps_b,
                                   double eps_p, double lam, double v_sites, double lgB, double* phi_hat, double* S,
                                   int* err, cudaStream_t s) {
  k_site_potentials<<<n, SITE_T, 0, s>>>(site, n, charges, nq, eps_b, eps_p, lam, v_sites, lgB, phi_hat, S, err);
  return cudaGetLastError();
}

cudaError_t launch_site_map(const double* site, int n, const double* phi_hat, const uint8_t* solvent, const Geom& g,
                            double ox, double oy, double oz, double h, double map_r, uint8_t* fixed, double* value,
                            cudaStream_t s) {
  k_site_map<<<blocks_for(g), FT, 0, s>>>(site, n, phi_hat, solvent, g, ox, oy, oz, h, map_r, fixed, value);
  return cudaGetLastError();
}

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
