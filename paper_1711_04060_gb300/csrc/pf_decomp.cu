// pf_decomp.cu -- the potential decomposition of Eqs. (5)-(10) on the device.  In the biomolecular (membrane)
// domain the potential is phi = phi~ + G with G = phi* + phi^L: phi* is the Coulomb potential of the fixed
// charges in a uniform dielectric eps_m (Eq. 6), phi^L the harmonic function that cancels phi* on the interface
// (Eqs. 9-10, with phi^L = -phi* there so that phi stays continuous), and phi~ solves the charge-free problem
// whose SMIB interface rows (Eqs. 16-18) carry the flux jump of G (Eq. 8) in place of the point charges.
//
// Discretisation (the choices the paper leaves open): the interface sits at the midpoint of every face between
// a membrane node and a solvent node; phi^L uses Shortley-Weller differences to those midpoints; on the x/y box
// sides dG/dn = 0, so phi~ keeps the plain mirror of Eq. (4); d phi^L/dn at a midpoint comes from the
// one-sided quadratic through the midpoint and two membrane nodes.  The Coulomb sums are evaluated directly
// (all charges at every point, FP64); the phi^L system has per-row coefficients, so it is stored as the seven
// diagonals of Section 4 and solved by a Jacobi-BiCGSTAB of its own.
#include "pf_decomp.cuh"
#include "pf_stencil.cuh"

namespace pf {
namespace {

constexpr int DT = NTHREADS;  // threads per block of the reduction kernels (the helpers of pf_stencil.cuh)

// phi* (k_BT/e) and, when grad != nullptr, its gradient at (x, y, z); err = 1 when a charge lies within 1e-6 h
__device__ void coulomb(const DecompArgs& a, double x, double y, double z, double* phi, double* grad) {
  double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  const double tiny = 1e-12 * a.h * a.h;
  for (int j = 0; j < a.nq; ++j) {
    const double dx = x - __ldg(a.ch + 4 * j), dy = y - __ldg(a.ch + 4 * j + 1), dz = z - __ldg(a.ch + 4 * j + 2);
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 < tiny) {
      atomicExch(a.err, 1);
      continue;
    }
    const double inv = 1.0 / sqrt(d2);
    const double q = __ldg(a.ch + 4 * j + 3);
    p += q * inv;
    if (grad) {
      const double q3 = q * inv * inv * inv;
      gx -= dx * q3;
      gy -= dy * q3;
      gz -= dz * q3;
    }
  }
  *phi = a.coef * p;
  if (grad) {
    grad[0] = a.coef * gx;
    grad[1] = a.coef * gy;
    grad[2] = a.coef * gz;
  }
}

#define PF_DROWS(g)                                                          \
  for (long row = blockIdx.x; row < (long)(g).ny * (g).nz; row += gridDim.x) \
    for (int i = threadIdx.x; i < (g).nx; i += blockDim.x)

__global__ void k_phiL_rows(DecompArgs a, double* A0, double* A1, double* A2, double* A3, double* A4, double* A5,
                            double* A6, double* b) {
  const Geom& g = a.g;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const uint8_t sc = a.solvent[c];
    // a side node and its mirror partner must be of the same kind: no interface across a mirror
    if ((i == 0 && g.nx > 1 && sc != a.solvent[c + 1]) || (i == g.nx - 1 && sc != a.solvent[c - 1]) ||
        (j == 0 && sc != a.solvent[c + g.px]) || (j == g.ny - 1 && sc != a.solvent[c - g.px]))
      atomicExch(a.err, 2);
    const double r[3] = {a.ox + a.h * i, a.oy + a.h * j, a.oz + a.h * k};
    double off[7] = {0, 0, 0, 0, 0, 0, 0};
    double diag = 0.0, rhs = 0.0;
    if (sc || k == 0 || k == g.nz - 1) {
      diag = 1.0;
      if (!sc) {  // G = 0 on the Dirichlet planes: phi^L = -phi*
        double p;
        coulomb(a, r[0], r[1], r[2], &p, nullptr);
        rhs = -p;
      }
    } else {
      const int idx[3] = {i, j, k}, n3[3] = {g.nx, g.ny, g.nz};
      const long st3[3] = {1, (long)g.px, g.plane};
      const double ih2 = 1.0 / (a.h * a.h);
      double grad[3];
      bool have_grad = false;
      for (int ax = 0; ax < 3; ++ax) {
        const int slot_lo = ax == 0 ? 2 : ax == 1 ? 3 : 5, slot_hi = ax == 0 ? 1 : ax == 1 ? 4 : 6;
        if (ax < 2 && (idx[ax] == 0 || idx[ax] == n3[ax] - 1)) {
          // box side: dG/dn = 0, the ghost value is partner + 2h d phi^L/dn = partner - 2h d phi*/dn
          const bool low = idx[ax] == 0;
          if (!have_grad) {
            double p;
            coulomb(a, r[0], r[1], r[2], &p, grad);
            have_grad = true;
          }
          const double nout = low ? -1.0 : 1.0;
          diag += 2.0 * ih2;
          off[low ? slot_hi : slot_lo] -= 2.0 * ih2;
          rhs += -2.0 * nout * grad[ax] / a.h;
          continue;
        }
        double hs[2], val[2];
        bool bnd[2];
        for (int sgn = 0; sgn < 2; ++sgn) {
          const long nb = c + (sgn ? st3[ax] : -st3[ax]);
          if (a.solvent[nb]) {
            double rx[3] = {r[0], r[1], r[2]};
            rx[ax] += (sgn ? 0.5 : -0.5) * a.h;
            double p;
            coulomb(a, rx[0], rx[1], rx[2], &p, nullptr);
            hs[sgn] = 0.5 * a.h;
            val[sgn] = -p;
            bnd[sgn] = true;
          } else {
            hs[sgn] = a.h;
            val[sgn] = 0.0;
            bnd[sgn] = false;
          }
        }
        for (int sgn = 0; sgn < 2; ++sgn) {
          const double cf = 2.0 / ((hs[0] + hs[1]) * hs[sgn]);
          diag += cf;
          if (bnd[sgn]) rhs += cf * val[sgn];
          else off[sgn ? slot_hi : slot_lo] -= cf;
        }
      }
    }
    A0[c] = diag;
    A1[c] = off[1];
    A2[c] = off[2];
    A3[c] = off[3];
    A4[c] = off[4];
    A5[c] = off[5];
    A6[c] = off[6];
    b[c] = rhs;
  }
}

struct Dia {
  const double* A[7];
};

// sum_d A_d[c] f(nb_d) over the neighbours that exist (the products with zero diagonals are skipped)
template <class F>
__device__ __forceinline__ double dia_row(const Dia& D, const Geom& g, long c, int i, int j, int k, F f) {
  double s = D.A[0][c] * f(c);
  if (i < g.nx - 1) s = fma(D.A[1][c], f(c + 1), s);
  if (i > 0) s = fma(D.A[2][c], f(c - 1), s);
  if (j > 0) s = fma(D.A[3][c], f(c - g.px), s);
  if (j < g.ny - 1) s = fma(D.A[4][c], f(c + g.px), s);
  if (k > 0) s = fma(D.A[5][c], f(c - g.plane), s);
  if (k < g.nz - 1) s = fma(D.A[6][c], f(c + g.plane), s);
  return s;
}

__device__ __forceinline__ bool identity_row(const Dia& D, long c) {
  return D.A[0][c] == 1.0 && D.A[1][c] == 0.0 && D.A[2][c] == 0.0 && D.A[3][c] == 0.0 && D.A[4][c] == 0.0 &&
         D.A[5][c] == 0.0 && D.A[6][c] == 0.0;
}

__global__ void k_dia_impose(Dia D, Geom g, const double* __restrict__ b, double* x) {
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    if (identity_row(D, c)) x[c] = b[c];
  }
}

__global__ void __launch_bounds__(DT) k_dia_start(Dia D, Geom g, const double* __restrict__ b,
                                                  const double* __restrict__ x, double* r, double* rt, double* p,
                                                  double* v, double tol, int max_iter, double* part, DiaState* st) {
  __shared__ double scratch[DT * 2];
  double rr = 0.0, bb = 0.0;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const double rc = b[c] - dia_row(D, g, c, i, j, k, [&](long q) { return x[q]; });
    r[c] = rc;
    rt[c] = rc;
    p[c] = 0.0;
    v[c] = 0.0;
    rr = fma(rc, rc, rr);
    bb = fma(b[c], b[c], bb);
  }
  double vals[2] = {rr, bb};
  block_partials<2>(vals, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[2];
  total_partials<2>(part, 0u, tot, scratch);
  if (threadIdx.x != 0) return;
  DiaState s{};
  s.bnorm2 = tot[1] > 0.0 ? tot[1] : 1.0;
  s.tol2 = tol * tol * s.bnorm2;
  s.rho = tot[0];
  s.rnorm2 = tot[0];
  s.max_iter = max_iter;
  s.done = tot[0] <= s.tol2 ? 1 : 0;
  *st = s;
}

// direction p' = r + beta (p - omega v) (formed at the node and its neighbours), v' = A M^-1 p', r~.v' -> alpha
__global__ void __launch_bounds__(DT) k_dia_dir(Dia D, Geom g, const double* __restrict__ r,
                                                const double* __restrict__ rt, const double* __restrict__ p,
                                                const double* __restrict__ v, double* pn, double* vn, double* part,
                                                DiaState* st) {
  __shared__ double scratch[DT];
  if (*(volatile int*)&st->done) return;
  const double be = st->beta, om = st->omega;
  auto dir = [&](long q) { return fma(be, fma(-om, v[q], p[q]), r[q]); };
  double a = 0.0;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    pn[c] = dir(c);
    const double vc = dia_row(D, g, c, i, j, k, [&](long q) { return dir(q) / D.A[0][q]; });
    vn[c] = vc;
    a = fma(rt[c], vc, a);
  }
  double vals[1] = {a};
  block_partials<1>(vals, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[1];
  total_partials<1>(part, 0u, tot, scratch);
  if (threadIdx.x != 0) return;
  st->ticket = 0;
  if (tot[0] == 0.0 || !isfinite(tot[0]) || !isfinite(st->rho / tot[0])) {
    st->status = 4;  // PF_E_BREAKDOWN
    st->done = 1;
    return;
  }
  st->alpha = st->rho / tot[0];
}

// s = r - alpha v', t = A M^-1 s and the inner products t.s, t.t, s.s, r~.s, r~.t -> omega, beta, the next rho
__global__ void __launch_bounds__(DT) k_dia_st(Dia D, Geom g, const double* __restrict__ r,
                                               const double* __restrict__ rt, const double* __restrict__ vn, double* t,
                                               double* part, DiaState* st) {
  __shared__ double scratch[DT * 5];
  if (*(volatile int*)&st->done) return;
  const double al = st->alpha;
  auto sv = [&](long q) { return fma(-al, vn[q], r[q]); };
  double ts = 0.0, tt = 0.0, ss = 0.0, rs = 0.0, rtt = 0.0;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const double sc = sv(c);
    const double tc = dia_row(D, g, c, i, j, k, [&](long q) { return sv(q) / D.A[0][q]; });
    t[c] = tc;
    ts = fma(tc, sc, ts);
    tt = fma(tc, tc, tt);
    ss = fma(sc, sc, ss);
    rs = fma(rt[c], sc, rs);
    rtt = fma(rt[c], tc, rtt);
  }
  double vals[5] = {ts, tt, ss, rs, rtt};
  block_partials<5>(vals, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[5];
  total_partials<5>(part, 0u, tot, scratch);
  if (threadIdx.x != 0) return;
  st->ticket = 0;
  if (tot[2] <= st->tol2) {  // early exit of the Templates algorithm: x += alpha M^-1 p, r = s
    st->sexit = 1;
    st->omega = 0.0;
    return;
  }
  if (tot[1] == 0.0 || !isfinite(tot[1]) || !isfinite(tot[0])) {
    st->status = 4;
    st->done = 1;
    return;
  }
  const double om = tot[0] / tot[1];
  const double rho_new = tot[3] - om * tot[4];
  st->omega = om;
  st->beta = om != 0.0 ? (rho_new / st->rho) * (st->alpha / om) : 0.0;
  st->rho = rho_new;
}

// x += alpha M^-1 p' + omega M^-1 s, r = s - omega t, ||r||^2 -> the stop test
__global__ void __launch_bounds__(DT) k_dia_x(Dia D, Geom g, double* r, const double* __restrict__ vn,
                                              const double* __restrict__ pn, const double* __restrict__ t, double* x,
                                              double* part, DiaState* st) {
  __shared__ double scratch[DT];
  if (*(volatile int*)&st->done) return;
  const double al = st->alpha, om = st->omega;
  const int sexit = st->sexit;
  double rr = 0.0;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const double di = 1.0 / D.A[0][c];
    const double sc = fma(-al, vn[c], r[c]);
    double xc = fma(al, pn[c] * di, x[c]);
    double rc = sc;
    if (!sexit) {
      xc = fma(om, sc * di, xc);
      rc = fma(-om, t[c], sc);
    }
    x[c] = xc;
    r[c] = rc;
    rr = fma(rc, rc, rr);
  }
  double vals[1] = {rr};
  block_partials<1>(vals, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[1];
  total_partials<1>(part, 0u, tot, scratch);
  if (threadIdx.x != 0) return;
  st->ticket = 0;
  st->iter += 1;
  st->rnorm2 = tot[0];
  if (sexit || tot[0] <= st->tol2) {
    st->done = 1;
    st->status = 0;
  } else if (st->omega == 0.0) {
    st->done = 1;
    st->status = 4;
  } else if (st->iter >= st->max_iter) {
    st->done = 1;
    st->status = 3;  // PF_E_NOCONV
  }
}

__global__ void k_decomp_G(DecompArgs a, const double* __restrict__ phiL, double* G) {
  const Geom& g = a.g;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    double p = 0.0;
    // every node is checked against the charges (a charge on a node has no finite G there)
    coulomb(a, a.ox + a.h * i, a.oy + a.h * j, a.oz + a.h * k, &p, nullptr);
    G[c] = a.solvent[c] ? 0.0 : p + phiL[c];
  }
}

__global__ void k_decomp_bif(DecompArgs a, const double* __restrict__ phiL, double* bif) {
  const Geom& g = a.g;
  PF_DROWS(g) {
    const long c = i + (long)g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    double acc = 0.0;
    if (k > 0 && k < g.nz - 1) {
      const int idx[3] = {i, j, k}, n3[3] = {g.nx, g.ny, g.nz};
      const long st3[3] = {1, (long)g.px, g.plane};
      const bool csol = a.solvent[c] != 0;
      for (int ax = 0; ax < 3; ++ax)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          const int in = idx[ax] + sgn;
          if (in < 0 || in >= n3[ax]) continue;
          const long nb = c + sgn * st3[ax];
          if ((a.solvent[nb] != 0) == csol) continue;
          const long cm = csol ? nb : c;
          const int nsgn = csol ? -sgn : sgn;  // n points from the membrane node to the solvent node
          const int im = csol ? in : idx[ax];  // index of cm along ax
          double xi[3] = {a.ox + a.h * i, a.oy + a.h * j, a.oz + a.h * k};
          xi[ax] += 0.5 * a.h * sgn;
          double p, gr[3];
          coulomb(a, xi[0], xi[1], xi[2], &p, gr);
          const double dstar = nsgn * gr[ax];
          const long cm2 = cm - nsgn * st3[ax];
          const bool inside = (nsgn > 0 ? im > 0 : im < n3[ax] - 1) && !a.solvent[cm2];
          const double f0 = -p, f1 = phiL[cm];
          const double dL = inside ? (8.0 * f0 - 9.0 * f1 + phiL[cm2]) / (3.0 * a.h) : (f0 - f1) / (0.5 * a.h);
          const double J = a.eps_m * (dstar + dL);
          acc += -(csol ? a.eps_s : a.eps_m) * J / ((a.eps_m + a.eps_s) * a.h);
        }
    }
    bif[c] = acc;
  }
}

__global__ void k_add_scale(const double* __restrict__ phi, const double* __restrict__ G, double scale,
                            double* out, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    out[c] = (G ? phi[c] + G[c] : phi[c]) * scale;
}

int row_grid(const Geom& g) {
  const long rows = (long)g.ny * g.nz;
  return (int)(rows < 2048 ? (rows > 0 ? rows : 1) : 2048);
}

Dia dia_of(const double* const A[7]) {
  Dia D;
  for (int d = 0; d < 7; ++d) D.A[d] = A[d];
  return D;
}

}  // namespace

cudaError_t launch_phiL_rows(const DecompArgs& a, double* const A[7], double* b, cudaStream_t s) {
  k_phiL_rows<<<row_grid(a.g), 128, 0, s>>>(a, A[0], A[1], A[2], A[3], A[4], A[5], A[6], b);
  return cudaGetLastError();
}

cudaError_t launch_dia_start(const double* const A[7], const DiaVecs& w, const Geom& g, double tol, int max_iter,
                             double* part, DiaState* st, cudaStream_t s) {
  const Dia D = dia_of(A);
  k_dia_impose<<<row_grid(g), 128, 0, s>>>(D, g, w.b, w.x);
  cudaMemsetAsync(&st->ticket, 0, sizeof(unsigned int), s);
  k_dia_start<<<row_grid(g), DT, 0, s>>>(D, g, w.b, w.x, w.r, w.rt, w.p[0], w.v[0], tol, max_iter, part, st);
  return cudaGetLastError();
}

cudaError_t launch_dia_iteration(const double* const A[7], const DiaVecs& w, int cur, const Geom& g, double* part,
                                 DiaState* st, cudaStream_t s) {
  const Dia D = dia_of(A);
  const int nxt = 1 - cur;
  k_dia_dir<<<row_grid(g), DT, 0, s>>>(D, g, w.r, w.rt, w.p[cur], w.v[cur], w.p[nxt], w.v[nxt], part, st);
  k_dia_st<<<row_grid(g), DT, 0, s>>>(D, g, w.r, w.rt, w.v[nxt], w.t, part, st);
  k_dia_x<<<row_grid(g), DT, 0, s>>>(D, g, w.r, w.v[nxt], w.p[nxt], w.t, w.x, part, st);
  return cudaGetLastError();
}

cudaError_t launch_decomp_G(const DecompArgs& a, const double* phiL, double* G, cudaStream_t s) {
  k_decomp_G<<<row_grid(a.g), 128, 0, s>>>(a, phiL, G);
  return cudaGetLastError();
}

cudaError_t launch_decomp_bif(const DecompArgs& a, const double* phiL, double* bif, cudaStream_t s) {
  k_decomp_bif<<<row_grid(a.g), 128, 0, s>>>(a, phiL, bif);
  return cudaGetLastError();
}

cudaError_t launch_add_scale(const double* phi, const double* G, double scale, double* out, long n, cudaStream_t s) {
  long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  k_add_scale<<<(int)(b < 1 ? 1 : b), 256, 0, s>>>(phi, G, scale, out, n);
  return cudaGetLastError();
}

}  // namespace pf
