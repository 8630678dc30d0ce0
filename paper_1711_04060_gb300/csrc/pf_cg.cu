// pf_cg.cu -- Jacobi-preconditioned conjugate gradients for the symmetric systems.
//
// Section 3 names the Laplace system (9) and PF1 (12) symmetric; with the zero-jump faces of
// Eqs. (15)-(18) the PF2 operator (13) is symmetric in the same sense.  The stored operators keep
// identity rows for fixed nodes and mirror ghosts on the x/y sides (Eq. 4), so A is symmetric only in
// the inner product <u, v>_w = sum_c w_c u_c v_c that weights a node by 1/2 for every x or y side it
// lies on (a mirror doubles a side row's coupling to its inner neighbour); with x = b on the identity
// rows, residuals and search directions vanish there.  Written with u = M p (M = diag A), one
// iteration is
//   u = r + beta u_old,  q = A M^-1 u,  alpha = <r, M^-1 r>_w / <M^-1 u, q>_w,
//   x += alpha M^-1 u,   r -= alpha q,  beta = <r', M^-1 r'>_w / <r, M^-1 r>_w,
// so the operator product has the form of the BiCGSTAB kernels: (A M^-1 u)_c = u_c - sum_nb f_nb
// dinv_nb u_nb on a free row (dinv = 0 marks identity rows, which drop out).  Two kernels per
// iteration: the direction with the operator product and <M^-1 u, q>_w, then the x / r update with
// <r, M^-1 r>_w and the norms of the stop test.  Neighbours are plain global loads (L1/L2 serve the
// reuse); each inner product is reduced by the last-arriving block over the block partials in fixed
// order, which also advances the scalars in the device state, so the host reads the state only every
// few iterations.
#include <math.h>

#include "pf_gb300.h"
#include "pf_cg.cuh"
#include "pf_stencil.cuh"

namespace pf {
namespace {

// Node t (0 <= t < nx ny nz, x fastest) -> its coordinates and its index in the padded layout.
struct Node {
  int i, j, k;
  long c;
};

__device__ __forceinline__ Node node_of(long t, const Geom& g) {
  Node n;
  n.i = (int)(t % g.nx);
  const long row = t / g.nx;
  n.j = (int)(row % g.ny);
  n.k = (int)(row / g.ny);
  n.c = n.i + (long)g.px * row;
  return n;
}

// 1/2 for every x or y side the node lies on
__device__ __forceinline__ double side_weight(const Node& n, const Geom& g) {
  const double wx = (n.i == 0 || n.i == g.nx - 1) ? 0.5 : 1.0;
  const double wy = (n.j == 0 || n.j == g.ny - 1) ? 0.5 : 1.0;
  return wx * wy;
}

// A free row: a non-zero Jacobi scaling on an interior plane (the Dirichlet planes are identity rows).
__device__ __forceinline__ bool free_row(const Node& n, const Geom& g, double di) {
  return di != 0.0 && n.k > 0 && n.k < g.nz - 1;
}

// The six neighbours of a free row (mirror images on the x/y sides) and their face coefficients.
struct Stencil {
  long e, w, n, s, u, d;
  double fe, fw, fn, fs, fu, fd;
};

__device__ __forceinline__ Stencil stencil_of(const CgOperator& a, const Geom& g, const Node& n) {
  Stencil st;
  const long c = n.c, sy = g.px, sz = g.plane;
  st.e = n.i < g.nx - 1 ? c + 1 : c - 1;
  st.w = n.i > 0 ? c - 1 : c + 1;
  st.n = n.j < g.ny - 1 ? c + sy : c - sy;
  st.s = n.j > 0 ? c - sy : c + sy;
  st.u = c + sz;
  st.d = c - sz;
  if (a.wE) {
    // the east (north) face of the last node in x (y) is the mirror face; the west (south) face of the
    // first node is its east (north) face
    st.fe = a.wE[c];
    st.fw = n.i > 0 ? a.wE[c - 1] : a.wE[c];
    st.fn = a.wN[c];
    st.fs = n.j > 0 ? a.wN[c - sy] : a.wN[c];
    st.fu = a.wU[c];
    st.fd = a.wU[c - sz];
  } else {
    st.fe = st.fw = st.fn = st.fs = st.fu = st.fd = a.wc;
  }
  return st;
}

constexpr int NV_START = 4, NV_DIR = 1, NV_UPD = 3;

// r = b - A x (u = 0 when u is given); the last block starts the state: ||b||^2, ||r||^2, max|r| and
// rho = <r, M^-1 r>_w, the REL2 threshold, and done when x already meets the stop test.
__global__ void __launch_bounds__(NTHREADS) k_cg_start(CgOperator a, Geom g, const double* __restrict__ b,
                                                       const double* __restrict__ x, double* __restrict__ r,
                                                       double* __restrict__ u, double* part, BicgState* st) {
  __shared__ double scratch[NTHREADS * NV_START];
  double bb = 0.0, rr = 0.0, rmax = 0.0, rz = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < g.n; t += (long)gridDim.x * blockDim.x) {
    const Node n = node_of(t, g);
    const double di = a.dinv[n.c];
    double rc;
    if (free_row(n, g, di)) {
      const Stencil s = stencil_of(a, g, n);
      double nb = s.fe * x[s.e];
      nb = fma(s.fw, x[s.w], nb);
      nb = fma(s.fn, x[s.n], nb);
      nb = fma(s.fs, x[s.s], nb);
      nb = fma(s.fu, x[s.u], nb);
      nb = fma(s.fd, x[s.d], nb);
      const double dg = a.diag ? a.diag[n.c] : a.diagc;
      rc = b[n.c] - fma(dg, x[n.c], -nb);
      rz = fma(side_weight(n, g) * rc * di, rc, rz);
    } else {
      rc = b[n.c] - x[n.c];
    }
    r[n.c] = rc;
    if (u) u[n.c] = 0.0;
    bb = fma(b[n.c], b[n.c], bb);
    rr = fma(rc, rc, rr);
    rmax = fmax(rmax, fabs(rc));
  }
  double v[NV_START] = {bb, rr, rmax, rz};
  block_partials<NV_START>(v, 4u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[NV_START];
  total_partials<NV_START>(part, 4u, tot, scratch);
  if (threadIdx.x == 0) {
    st->bnorm2 = tot[0];
    st->rnorm2 = tot[1];
    st->rinf = tot[2];
    st->rho = tot[3];
    st->alpha = 0.0;
    st->beta = 0.0;
    st->iter = 0;
    st->tol2 = st->tol * st->tol * (tot[0] > 0.0 ? tot[0] : 1.0);
    const bool conv = st->norm == PF_NORM_REL2 ? tot[1] <= st->tol2 : tot[2] < st->tol;
    if (conv) {
      st->status = PF_OK;
      st->done = 1;
    } else if (!(tot[3] > 0.0)) {  // a residual on rows whose Jacobi scaling is not positive
      st->status = PF_E_BREAKDOWN;
      st->done = 1;
    } else if (st->max_iter < 1) {
      st->status = PF_E_NOCONV;
      st->done = 1;
    }
    st->ticket = 0;
  }
}

// u = r + beta u_old (written to un), q = A M^-1 u; the last block sets alpha = rho / <M^-1 u, q>_w.
__global__ void __launch_bounds__(NTHREADS) k_cg_direction(CgOperator a, Geom g, const double* __restrict__ r,
                                                           const double* __restrict__ uo, double* __restrict__ un,
                                                           double* __restrict__ q, double* part, BicgState* st) {
  __shared__ double scratch[NTHREADS * NV_DIR];
  if (*(volatile int*)&st->done) return;
  const double beta = st->beta;
  double pq = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < g.n; t += (long)gridDim.x * blockDim.x) {
    const Node n = node_of(t, g);
    const double di = a.dinv[n.c];
    const double uc = fma(beta, uo[n.c], r[n.c]);
    double qc = uc;
    if (free_row(n, g, di)) {
      const Stencil s = stencil_of(a, g, n);
      double nb = s.fe * (a.dinv[s.e] * fma(beta, uo[s.e], r[s.e]));
      nb = fma(s.fw, a.dinv[s.w] * fma(beta, uo[s.w], r[s.w]), nb);
      nb = fma(s.fn, a.dinv[s.n] * fma(beta, uo[s.n], r[s.n]), nb);
      nb = fma(s.fs, a.dinv[s.s] * fma(beta, uo[s.s], r[s.s]), nb);
      nb = fma(s.fu, a.dinv[s.u] * fma(beta, uo[s.u], r[s.u]), nb);
      nb = fma(s.fd, a.dinv[s.d] * fma(beta, uo[s.d], r[s.d]), nb);
      qc = uc - nb;
      pq = fma(side_weight(n, g) * di * uc, qc, pq);
    }
    un[n.c] = uc;
    q[n.c] = qc;
  }
  double v[NV_DIR] = {pq};
  block_partials<NV_DIR>(v, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[NV_DIR];
  total_partials<NV_DIR>(part, 0u, tot, scratch);
  if (threadIdx.x == 0) {
    if (tot[0] > 0.0) {
      st->alpha = st->rho / tot[0];
    } else {  // p.Ap <= 0: the operator is not positive definite on this direction
      st->status = PF_E_BREAKDOWN;
      st->done = 1;
    }
    st->ticket = 0;
  }
}

// x += alpha M^-1 u, r -= alpha q; the last block counts the iteration, applies the stop test and sets
// beta and the next rho.
__global__ void __launch_bounds__(NTHREADS) k_cg_update(CgOperator a, Geom g, const double* __restrict__ un,
                                                        const double* __restrict__ q, double* __restrict__ x,
                                                        double* __restrict__ r, double* part, BicgState* st) {
  __shared__ double scratch[NTHREADS * NV_UPD];
  if (*(volatile int*)&st->done) return;
  const double alpha = st->alpha;
  double rr = 0.0, rmax = 0.0, rz = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < g.n; t += (long)gridDim.x * blockDim.x) {
    const Node n = node_of(t, g);
    const double di = a.dinv[n.c];
    const double rc = fma(-alpha, q[n.c], r[n.c]);
    x[n.c] = fma(alpha, di * un[n.c], x[n.c]);
    r[n.c] = rc;
    rr = fma(rc, rc, rr);
    rmax = fmax(rmax, fabs(rc));
    if (free_row(n, g, di)) rz = fma(side_weight(n, g) * rc * di, rc, rz);
  }
  double v[NV_UPD] = {rr, rmax, rz};
  block_partials<NV_UPD>(v, 2u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[NV_UPD];
  total_partials<NV_UPD>(part, 2u, tot, scratch);
  if (threadIdx.x == 0) {
    const int it = st->iter + 1;
    st->iter = it;
    st->rnorm2 = tot[0];
    st->rinf = tot[1];
    const bool conv = st->norm == PF_NORM_REL2 ? tot[0] <= st->tol2 : tot[1] < st->tol;
    if (conv) {
      st->status = PF_OK;
      st->done = 1;
    } else if (it >= st->max_iter) {
      st->status = PF_E_NOCONV;
      st->done = 1;
    } else if (!(tot[2] > 0.0)) {
      st->status = PF_E_BREAKDOWN;
      st->done = 1;
    } else {
      st->beta = tot[2] / st->rho;
      st->rho = tot[2];
    }
    st->ticket = 0;
  }
}

// one thread per node, at most as many blocks as the partials buffer holds
int cg_blocks(const Geom& g) {
  const long want = (g.n + NTHREADS - 1) / NTHREADS;
  const int cap = max_partial_blocks();
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_cg_start(const CgOperator& a, const Geom& g, const double* b, const double* x, double* r,
                            double* u, double* part, BicgState* st, cudaStream_t s) {
  k_cg_start<<<cg_blocks(g), NTHREADS, 0, s>>>(a, g, b, x, r, u, part, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_direction(const CgOperator& a, const Geom& g, const double* r, const double* uo, double* un,
                                double* q, double* part, BicgState* st, cudaStream_t s) {
  k_cg_direction<<<cg_blocks(g), NTHREADS, 0, s>>>(a, g, r, uo, un, q, part, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(const CgOperator& a, const Geom& g, const double* un, const double* q, double* x,
                             double* r, double* part, BicgState* st, cudaStream_t s) {
  k_cg_update<<<cg_blocks(g), NTHREADS, 0, s>>>(a, g, un, q, x, r, part, st);
  return cudaGetLastError();
}

}  // namespace pf
