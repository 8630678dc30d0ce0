// pf_kernels.cu -- sm_103a kernels of the Poisson-Fermi hot path on one grid: the single-grid stencil
// launches (BiCGSTAB phases and the FP64 residual, whose body is in pf_stencil.cuh), operator setup, the
// pointwise Fermi/steric step of Eq. (1), the right-hand-side builds, relaxation and the elementwise
// helpers of the solver, with their host launchers.
#include <math.h>
#include <stdio.h>

#include "pf_df.cuh"
#include "pf_stencil.cuh"

namespace pf {

int tiles_for(int nx, int ny, int nz, int zc, int edges) {
  const int ntx = tiles_x(nx, edges), nty = tiles_y(ny, edges), nzc = (nz - 2 + zc - 1) / zc;
  return ntx * nty * nzc;
}

// ------------------------------------------------------------------ single-grid stencil kernel
// One grid: a persistent launch whose blocks stride over the grid's tiles.
template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB) k_stencil(const __grid_constant__ Maps<Op::NH, Op::NC> maps,
                                                      typename Op::Args a, Geom g, int ntiles,
                                                      unsigned long long wait_limit) {
  stencil_run<Op>(&maps, a, g, ntiles, blockIdx.x, gridDim.x, wait_limit);
}

// ------------------------------------------------------------------ elementwise kernels
// Nodes are visited row by row: row r = j + ny*k holds i = 0..nx-1 at padded index i + px*r.
#define PF_ROWS(g)                                                           \
  for (long row = blockIdx.x; row < (long)(g).ny * (g).nz; row += gridDim.x) \
    for (int i = threadIdx.x; i < (g).nx; i += blockDim.x)

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_init_zero(const T* __restrict__ b, Geom g, T* __restrict__ r,
                                                        T* __restrict__ rt, T* __restrict__ p, T* __restrict__ v,
                                                        T* __restrict__ t, double* part, BicgState* st) {
  __shared__ double scratch[NTHREADS * 2];
  Acc<T> abb;
  T bmax = T(0);
  for (long row = blockIdx.x; row < (long)g.ny * g.nz; row += gridDim.x) {
    const long k = row / g.ny;
    if (k == 0 || k == g.nz - 1) continue;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const long c = i + (long)g.px * row;
      const T bc = b[c];
      r[c] = bc;
      rt[c] = bc;
      p[c] = T(0);
      v[c] = T(0);
      t[c] = T(0);
      abb.prod(bc, bc);
      bmax = fmax(bmax, tabs(bc));
    }
  }
  double vals[2] = {abb.value(), (double)bmax};
  block_partials<2>(vals, 2u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[2];
  total_partials<2>(part, 2u, tot, scratch);
  if (threadIdx.x != 0) return;
  double bb = tot[0] + st->bnorm2;
  if (bb == 0.0) bb = 1.0;
  st->bnorm2 = bb;
  st->rho = tot[0];
  st->rnorm2 = tot[0];
  st->rinf = tot[1];
  set_tol2(st, tot[0], bb);
  st->alpha = st->omega = st->beta = 0.0;
  st->sexit = 0;
  st->iter = 0;
  st->status = 0;
  st->done = (st->norm == 0 ? (tot[0] <= st->tol2) : (tot[1] < st->tol)) ? 1 : 0;
  st->ticket = 0;
}

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

// Harmonic face coefficients (Eqs. 15-18 with zero jump) over h^2 for the east, north and up faces of
// every node; at i = nx-1 (j = ny-1) the east (north) face is the mirror face to the ghost node.
// dsum = sum of the six faces (the diagonal of -div(eps grad)), 1 on the Dirichlet planes.
__global__ void k_faces(const double* __restrict__ eps, Geom g, double ih2, double* wE, double* wN, double* wU,
                        double* dsum, float* gh32) {
  const long sy = g.px, sz = g.plane;
  PF_ROWS(g) {
    const long c = i + g.px * row;
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const double e = eps[c];
    const double fe = __dmul_rn(harm(e, eps[i < g.nx - 1 ? c + 1 : c - 1]), ih2);
    const double fw = __dmul_rn(harm(e, eps[i > 0 ? c - 1 : c + 1]), ih2);
    const double fn = __dmul_rn(harm(e, eps[j < g.ny - 1 ? c + sy : c - sy]), ih2);
    const double fs = __dmul_rn(harm(e, eps[j > 0 ? c - sy : c + sy]), ih2);
    const double fu = k < g.nz - 1 ? __dmul_rn(harm(e, eps[c + sz]), ih2) : 0.0;
    const double fd = k > 0 ? __dmul_rn(harm(e, eps[c - sz]), ih2) : 0.0;
    wE[c] = fe;
    wN[c] = fn;
    wU[c] = fu;
    // summation order of the assembled diagonal: east, west, north, south, up, down
    double d = __dadd_rn(fe, fw);
    d = __dadd_rn(d, fn);
    d = __dadd_rn(d, fs);
    d = __dadd_rn(d, fu);
    d = __dadd_rn(d, fd);
    dsum[c] = (k == 0 || k == g.nz - 1) ? 1.0 : d;
    gh32[c] = (float)(0.5 / (e * ih2));
  }
}

// Trilinear spreading of the fixed charges (Eq. 3 on the grid): one thread, charges in order.
__global__ void k_spread(const double* __restrict__ ch, int nq, double ox, double oy, double oz, double h, double lam,
                         Geom g, double* f, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double org[3] = {ox, oy, oz};
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int q = 0; q < nq; ++q) {
    int i0[3];
    double tt[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      const double gg = __ddiv_rn(__dsub_rn(ch[4 * q + a], org[a]), h);
      int i = (int)floor(gg);
      if (i == n[a] - 1 && gg == (double)(n[a] - 1)) i = n[a] - 2;
      if (!(gg >= 0.0) || i < 0 || i > n[a] - 2) ok = false;
      i0[a] = i;
      tt[a] = __dsub_rn(gg, (double)i);
    }
    if (!ok) {
      *err = 1;
      return;
    }
    const double amp = __ddiv_rn(__dmul_rn(lam, ch[4 * q + 3]), __dmul_rn(__dmul_rn(h, h), h));
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
      const double w = __dmul_rn(__dmul_rn(dx ? tt[0] : __dsub_rn(1.0, tt[0]), dy ? tt[1] : __dsub_rn(1.0, tt[1])),
                                 dz ? tt[2] : __dsub_rn(1.0, tt[2]));
      const long id = (i0[0] + dx) + (long)g.px * ((i0[1] + dy) + (long)g.ny * (i0[2] + dz));
      f[id] = __dadd_rn(f[id], __dmul_rn(amp, w));
    }
  }
}

__global__ void k_eps_diag(const double* __restrict__ dsum, const double* __restrict__ sig,
                           const uint8_t* __restrict__ smask, Geom g, double* diag, double* dinv, float* dinv32) {
  PF_ROWS(g) {
    const long c = i + g.px * row;
    const long k = row / g.ny;
    double d = 1.0, di = 0.0;
    if (k > 0 && k < g.nz - 1) {
      d = dsum[c];
      if (sig && (!smask || smask[c])) d = __dadd_rn(d, sig[c]);
      di = 1.0 / d;
    }
    diag[c] = d;
    dinv[c] = di;
    if (dinv32) dinv32[c] = (float)di;
  }
}

__global__ void k_pf1_dinv(const uint8_t* __restrict__ solvent, Geom g, double dinvc, double* dinv, float* dinv32) {
  PF_ROWS(g) {
    const long c = i + g.px * row;
    const long k = row / g.ny;
    const double di = (k > 0 && k < g.nz - 1 && solvent[c]) ? dinvc : 0.0;
    dinv[c] = di;
    if (dinv32) dinv32[c] = (float)di;
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    b[c] = (float)a[c];
}

__global__ void k_impose(double* __restrict__ x, const double* __restrict__ b, const double* __restrict__ dinv,
                         long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    if (dinv[c] == 0.0) x[c] = b[c];
}

__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ d, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    x[c] += (double)d[c];
}

__global__ void k_pack_d(const double* __restrict__ src, double* __restrict__ dst, Geom g) {
  PF_ROWS(g) dst[i + g.px * row] = src[i + (long)g.nx * row];
}

__global__ void k_pack_u8(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, Geom g) {
  PF_ROWS(g) dst[i + g.px * row] = src[i + (long)g.nx * row];
}

__global__ void k_unpack(const double* __restrict__ src, double* __restrict__ dst, Geom g, int count) {
  for (int f = 0; f < count; ++f) {
    const double* s = src + f * g.np;
    double* d = dst + f * g.n;
    PF_ROWS(g) d[i + (long)g.nx * row] = s[i + g.px * row];
  }
}

// b.b over the two Dirichlet planes (which the stencil kernels do not visit) -> st->bnorm2: blocks take
// rows of the two planes in turn, the last-arriving block sums the block partials in fixed order.
__global__ void __launch_bounds__(NTHREADS) k_plane_bb(const double* __restrict__ b, Geom g, double* part,
                                                       BicgState* st) {
  __shared__ double scratch[NTHREADS];
  double a = 0.0;
  const long last = g.plane * (g.nz - 1);
  for (long row = blockIdx.x; row < 2L * g.ny; row += gridDim.x) {
    const long base = (row < g.ny ? 0 : last) + g.px * (row % g.ny);
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const double u = b[base + i];
      a = fma(u, u, a);
    }
  }
  double vals[1] = {a};
  block_partials<1>(vals, 0u, part, scratch);
  if (!arrive_last(&st->ticket)) return;
  double tot[1];
  total_partials<1>(part, 0u, tot, scratch);
  if (threadIdx.x == 0) {
    st->bnorm2 = tot[0];
    st->ticket = 0;
  }
}

// keep_r0 != 0 keeps r0norm2 and bnorm2 of the previous state (the same right-hand side)
__global__ void k_set_state(BicgState* st, double tol, int norm, int max_iter, double tol_r0, int keep_r0) {
  const double r0 = keep_r0 ? st->r0norm2 : -1.0;
  const double b0 = keep_r0 ? st->bnorm2 : 0.0;
  BicgState s = {};
  s.tol = tol;
  s.norm = norm;
  s.max_iter = max_iter;
  s.tol_r0 = tol_r0;
  s.r0norm2 = r0;
  s.bnorm2 = b0;
  *st = s;
}


// ------------------------------------------------------------------ Eq. (1) pointwise step
// With la_i = ln(v_i cB_i) - z_i phi - p_i ln Gamma^B, the void fraction Gamma = e^u solves
//   f(u) = e^u + sum_i exp(la_i + p_i u) - 1 = 0,
// f increasing; every term is at most 1 on the bracket [lo, hi] below, so nothing overflows there.
// Newton runs first in FP32 on du = u - u0 (u0: the previous outer iterate's root, or ln Gamma^B), then in
// FP64 until the Newton step du is below 1e-6 max(1, |u|); Newton converges quadratically (f''/f' is at
// most max p_i), so u + du is within about p du^2 / 2 <= 1e-12 max(1, u^2) of the root, and the
// concentrations come from the last FP64 terms, term_i = v_i C_i, moved to u + du by
// exp(p_i du) = 1 + p_i du + (p_i du)^2/2.  The FP32 phase leaves |du| near FP32 rounding, so one FP64
// evaluation usually suffices.
struct FermiOut {
  double u, S, G;
  double C[MAXSP];
};

__device__ __forceinline__ bool fermi_point(const SpeciesParams& sp, double phi, double u0, FermiOut& o) {
  double la[MAXSP];
  double hi = 0.0, lo = -sp.lnn;
  for (int i = 0; i < sp.ns; ++i) {
    la[i] = sp.lvc[i] - sp.z[i] * phi - sp.p[i] * sp.lgB;
    if (!(sp.lvc[i] > -INFINITY)) continue;
    hi = fmin(hi, -la[i] * sp.inv_p[i]);
    lo = fmin(lo, (-la[i] - sp.lnn) * sp.inv_p[i]);
  }
  double u = u0;
  if (!(u < hi && u > lo)) u = 0.5 * (lo + hi);
  // FP32 phase on du = u - u0c (u0c: the clamped start)
  {
    const double uc = u;
    float A[MAXSP];
    for (int i = 0; i < sp.ns; ++i) A[i] = (sp.lvc[i] > -INFINITY) ? (float)(la[i] + sp.p[i] * uc) : -INFINITY;
    const float Ae = (float)uc;
    float du = 0.f, dlo = (float)(lo - uc), dhi = (float)(hi - uc);
    for (int it = 0; it < 60; ++it) {
      const float eu = __expf(Ae + du);
      float f = eu - 1.f, df = eu;
      for (int i = 0; i < sp.ns; ++i) {
        const float pi = (float)sp.p[i];
        const float term = __expf(A[i] + pi * du);
        f += term;
        df = fmaf(pi, term, df);
      }
      if (f > 0.f) dhi = du; else dlo = du;
      float dn = du - f / df;
      if (!(dn > dlo && dn < dhi)) dn = 0.5f * (dlo + dhi);
      const float step = dn - du;
      du = dn;
      if (fabsf(step) <= 2e-6f * fmaxf(1.f, fabsf((float)uc + du))) break;
    }
    u = uc + (double)du;
    if (!(u < hi && u > lo)) u = 0.5 * (lo + hi);
  }
  // FP64 phase
  double term[MAXSP];
  for (int it = 0; it < 200; ++it) {
    const double eu = exp(u);
    double f = eu - 1.0, df = eu;
    for (int i = 0; i < sp.ns; ++i) {
      term[i] = (sp.lvc[i] > -INFINITY) ? exp(la[i] + sp.p[i] * u) : 0.0;
      f += term[i];
      df += sp.p[i] * term[i];
    }
    const double du = (f == 0.0) ? 0.0 : -f / df;
    if (fabs(du) <= 1e-6 * fmax(1.0, fabs(u))) {  // converged: take the last Newton step and finish
      const double un = u + du;
      o.u = un;
      o.S = un - sp.lgB;
      o.G = eu * (1.0 + du + 0.5 * du * du);
      for (int i = 0; i < sp.ns; ++i) {
        const double x = sp.p[i] * du;
        o.C[i] = term[i] * sp.inv_v[i] * (1.0 + x + 0.5 * x * x);
      }
      return isfinite(un);
    }
    if (f > 0.0) hi = u; else lo = u;
    double un = u + du;
    if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);  // safeguard: bisect
    u = un;
  }
  return false;
}

// ulast holds each node's ln Gamma from the previous call (warm != 0; from u32start when that is given) and
// receives the new one.
__global__ void k_fermi(const double* __restrict__ phi0, const uint8_t* __restrict__ solvent,
                        const double* __restrict__ ffix, SpeciesParams sp, Geom g, double* b1, double* sig, double* c2,
                        double* C, double* S, double* G, double* ulast, int warm, int* err,
                        const float* __restrict__ u32start) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < g.np; c += (long)gridDim.x * blockDim.x) {
    const long row = c / g.px;
    const int i = (int)(c - row * g.px);
    if (i >= g.nx) continue;  // pad column
    const long k = row / g.ny;
    const double ph = phi0[c];
    const bool sol = solvent[c] != 0;
    FermiOut fo;
    bool ok = false;
    if (sol) {
      ok = fermi_point(sp, ph, warm ? (u32start ? (double)u32start[c] : ulast[c]) : sp.lgB, fo);
      if (!ok) atomicExch(err, 5);
      else ulast[c] = fo.u;
    }
    double rho = 0.0, kap = 0.0;
    for (int s = 0; s < sp.ns; ++s) {
      const double Ci = (sol && ok) ? fo.C[s] : 0.0;
      rho += sp.z[s] * Ci;
      kap += sp.lam * sp.z[s] * sp.z[s] * Ci;
      if (C) C[s * g.np + c] = Ci;
    }
    if (b1) b1[c] = (sol && k > 0 && k < g.nz - 1) ? -sp.lam * rho : 0.0;
    if (sig) sig[c] = kap;
    if (c2) c2[c] = fma(kap, ph, ffix[c]);
    if (S) S[c] = (sol && ok) ? fo.S : 0.0;
    if (G) G[c] = (sol && ok) ? fo.G : 0.0;
  }
}

// ------------------------------------------------------------------ Eq. (1) in double-float arithmetic
// The same root and Newton finish as fermi_point, with every operation on the FP32 pipes: the bracket and
// the FP32 Newton phase as there, then Newton steps in double-float (hi + lo pairs, about 48 bits) until the
// step is below 1e-6 max(1, |u|); the terms term_i = v_i C_i come from df_exp to about 1e-14 relative and
// are moved to the finished root by exp(p_i du) = 1 + p_i du + (p_i du)^2 / 2 like the FP64 form.
struct FermiDF {
  dfl u;
  dfl C[MAXSP];  // A^-3
};

__device__ __forceinline__ bool fermi_point_df(const SpeciesDF& sp, dfl phi, float u0, const float* thi,
                                               const float* tlo, FermiDF& o) {
  dfl la[MAXSP];
  float hi = 0.0f, lo = -sp.lnn;
#pragma unroll
  for (int i = 0; i < MAXSP; ++i) {
    if (i >= sp.ns) break;
    la[i] = df_add({sp.chi[i], sp.clo[i]}, df_mul_f(phi, -sp.z[i]));
    if (!sp.present[i]) continue;
    hi = fminf(hi, -la[i].hi * sp.inv_p[i]);
    lo = fminf(lo, (-la[i].hi - sp.lnn) * sp.inv_p[i]);
  }
  float uc = u0;
  if (!(uc < hi && uc > lo)) uc = 0.5f * (lo + hi);
  // FP32 phase on du = u - uc: the exponents la_i + p_i uc are formed in double-float and rounded once
  float A[MAXSP];
#pragma unroll
  for (int i = 0; i < MAXSP; ++i) {
    if (i >= sp.ns) break;
    const dfl x = df_add(la[i], df_mul_f({sp.phi[i], sp.plo[i]}, uc));
    A[i] = sp.present[i] ? x.hi + x.lo : -INFINITY;
  }
  float du = 0.f, dlo = lo - uc, dhi = hi - uc;
  for (int it = 0; it < 60; ++it) {
    const float eu = __expf(uc + du);
    float f = eu - 1.f, dfd = eu;
#pragma unroll
    for (int i = 0; i < MAXSP; ++i) {
      if (i >= sp.ns) break;
      const float term = __expf(A[i] + sp.phi[i] * du);
      f += term;
      dfd = fmaf(sp.phi[i], term, dfd);
    }
    if (f > 0.f) dhi = du; else dlo = du;
    float dn = du - __fdividef(f, dfd);
    if (!(dn > dlo && dn < dhi)) dn = 0.5f * (dlo + dhi);
    const float step = dn - du;
    du = dn;
    if (fabsf(step) <= 2e-6f * fmaxf(1.f, fabsf(uc + du))) break;
  }
  dfl u = two_sum(uc, du);
  float blo = lo, bhi = hi;
  // double-float Newton phase
  for (int it = 0; it < 8; ++it) {
    const dfl eu = df_exp(u, thi, tlo);
    dfl f = df_add_f(eu, -1.0f);
    float dfd = eu.hi;
    dfl t[MAXSP];
#pragma unroll
    for (int i = 0; i < MAXSP; ++i) {
      if (i >= sp.ns) break;
      t[i] = {0.f, 0.f};
      if (!sp.present[i]) continue;
      t[i] = df_exp(df_add(la[i], df_mul({sp.phi[i], sp.plo[i]}, u)), thi, tlo);
      f = df_add(f, t[i]);
      dfd = fmaf(sp.phi[i], t[i].hi, dfd);
    }
    const float d = -(f.hi + f.lo) / dfd;
    if (fabsf(d) <= 1e-6f * fmaxf(1.f, fabsf(u.hi))) {  // converged: finish with this Newton step
      o.u = df_add_f(u, d);
#pragma unroll
      for (int i = 0; i < MAXSP; ++i) {
        if (i >= sp.ns) break;
        const float x = sp.phi[i] * d;
        const dfl corr = fast_two_sum(1.0f, fmaf(0.5f * x, x, x));
        o.C[i] = df_mul(df_mul(t[i], {sp.ivhi[i], sp.ivlo[i]}), corr);
      }
      return isfinite(o.u.hi);
    }
    if (f.hi > 0.f) bhi = u.hi; else blo = u.hi;
    dfl un = df_add_f(u, d);
    if (!(un.hi > blo && un.hi < bhi)) un = {0.5f * (blo + bhi), 0.f};  // safeguard: bisect
    u = un;
  }
  return false;
}

// Splits a finite double into a double-float pair (hi: nearest float, lo: nearest float to the rest).
__device__ __forceinline__ dfl split_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

__global__ void __launch_bounds__(256, 3) k_fermi_df(const double* __restrict__ phi0, const uint8_t* __restrict__ solvent,
                                                  const double* __restrict__ ffix, SpeciesDF sp, Exp2Table tab, Geom g,
                                                  double* b1, double* sig, double* c2, float* u32, int warm, int* err) {
  __shared__ float thi[64], tlo[64];
  if (threadIdx.x < 64) {
    thi[threadIdx.x] = tab.hi[threadIdx.x];
    tlo[threadIdx.x] = tab.lo[threadIdx.x];
  }
  __syncthreads();
  const dfl lam = {sp.lamhi, sp.lamlo};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < g.np; c += (long)gridDim.x * blockDim.x) {
    const long row = c / g.px;
    const int i = (int)(c - row * g.px);
    if (i >= g.nx) continue;  // pad column
    const long k = row / g.ny;
    const double ph = phi0[c];
    if (!solvent[c]) {
      b1[c] = 0.0;
      sig[c] = 0.0;
      c2[c] = ffix[c];
      continue;
    }
    FermiDF fo;
    const bool ok = fermi_point_df(sp, split_double(ph), warm ? u32[c] : sp.lgB, thi, tlo, fo);
    dfl rho = {0.f, 0.f};
    float kap = 0.f;
    if (ok) {
      u32[c] = fo.u.hi;
#pragma unroll
      for (int s = 0; s < MAXSP; ++s) {
        if (s >= sp.ns) break;
        rho = df_add(rho, df_mul_f(fo.C[s], sp.z[s]));
        kap = fmaf(sp.z[s] * sp.z[s], fo.C[s].hi, kap);
      }
      kap *= sp.lamhi;
    } else {
      atomicExch(err, 5);
    }
    const double kd = (double)kap;
    b1[c] = (k > 0 && k < g.nz - 1) ? -df_to_double(df_mul(lam, rho)) : 0.0;
    sig[c] = kd;
    c2[c] = fma(kd, ph, ffix[c]);
  }
}

SpeciesDF species_df(const SpeciesParams& sp) {
  SpeciesDF d{};
  d.ns = sp.ns;
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  for (int i = 0; i < sp.ns; ++i) {
    d.present[i] = sp.lvc[i] > -INFINITY ? 1 : 0;
    d.z[i] = (float)sp.z[i];
    split(sp.p[i], d.phi[i], d.plo[i]);
    d.inv_p[i] = (float)sp.inv_p[i];
    split(d.present[i] ? sp.lvc[i] - sp.p[i] * sp.lgB : -200.0, d.chi[i], d.clo[i]);
    split(sp.inv_v[i], d.ivhi[i], d.ivlo[i]);
  }
  d.lnn = (float)sp.lnn;
  d.lgB = (float)sp.lgB;
  split(sp.lam, d.lamhi, d.lamlo);
  return d;
}

__global__ void k_pf2_rhs(const double* __restrict__ psi, const uint8_t* __restrict__ solvent,
                          const double* __restrict__ c2, double eps_s, double lo, double hi, Geom g, double* b2) {
  PF_ROWS(g) {
    const long c = i + g.px * row;
    const long k = row / g.ny;
    double v;
    if (k == 0) v = lo;
    else if (k == g.nz - 1) v = hi;
    else v = (solvent[c] ? -eps_s * psi[c] : 0.0) + c2[c];
    b2[c] = v;
  }
}

__global__ void __launch_bounds__(NTHREADS) k_relax(double* __restrict__ phi0, const double* __restrict__ phi,
                                                    double omega, long n, double* part, unsigned int* ticket,
                                                    double* delta) {
  __shared__ double scratch[NTHREADS];
  double m = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double o = phi0[c];
    const double nw = omega * o + (1.0 - omega) * phi[c];
    m = fmax(m, fabs(nw - o));
    phi0[c] = nw;
  }
  double vals[1] = {m};
  block_partials<1>(vals, 1u, part, scratch);
  if (!arrive_last(ticket)) return;
  double tot[1];
  total_partials<1>(part, 1u, tot, scratch);
  if (threadIdx.x == 0) {
    *delta = tot[0];
    *ticket = 0;
  }
}

__global__ void k_scale(const double* __restrict__ a, double s, double* __restrict__ out, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    out[c] = a[c] * s;
}

__global__ void k_set_dirichlet(double* x, double lo, double hi, Geom g) {
  const long last = g.plane * (g.nz - 1);
  for (long r = blockIdx.x; r < g.ny; r += gridDim.x)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      x[i + g.px * r] = lo;
      x[last + i + g.px * r] = hi;
    }
}

// ------------------------------------------------------------------ launchers
static int g_nsm = 0;
static int nsm() {
  if (!g_nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (g_nsm <= 0) g_nsm = 1;
  }
  return g_nsm;
}

int max_partial_blocks() { return nsm() * 16 > 2048 ? nsm() * 16 : 2048; }

static int ew_blocks(long n) {
  long b = (n + 255) / 256;
  const long cap = (long)nsm() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// At least three waves of the FP32 phase kernels (four blocks per SM) with the narrow tiles: below that the
// narrow tiles run beside the full ones and taking them into the edge tiles only lengthens those.
int edges_for(int nx, int ny, int nz) { return tiles_for(nx, ny, nz, ZC, 0) >= 3 * 4 * nsm() ? 1 : 0; }

static int row_blocks(const Geom& g) {
  long b = (long)g.ny * g.nz;
  const long cap = (long)nsm() * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

bool encode_map(CUtensorMap* m, const void* base, const Geom& g, int elem_bytes, int box_kind) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.px * elem_bytes, (cuuint64_t)g.plane * elem_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)HBX, (cuuint32_t)(box_kind == BOX_HALO ? HBY : TY), 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Grid size of a stencil kernel: every SM, as many blocks as fit (shared memory, registers), never
// more blocks than tiles.  Raises the kernel's dynamic shared-memory limit on first use.
template <class Op>
static int stencil_blocks(int ntiles) {
  static int per_sm = 0;
  if (!per_sm) {
    const int bytes = smem_bytes<Op>();
    cudaFuncSetAttribute(k_stencil<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_stencil<Op>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_stencil<Op>, NTHREADS, bytes);
    per_sm = o > 0 ? o : 1;
  }
  const int b = nsm() * per_sm;
  return b < ntiles ? b : ntiles;
}

template <class Op>
static cudaError_t launch_stencil(const Maps<Op::NH, Op::NC>& m, const typename Op::Args& a, const Geom& g,
                                  const Launch& L) {
  static_assert(scratch_fits<Op>(), "reduction scratch must fit in the stage ring");
  const int blocks = stencil_blocks<Op>(L.ntiles);
  k_stencil<Op><<<blocks, NTHREADS, smem_bytes<Op>(), L.stream>>>(m, a, g, L.ntiles, L.wait_limit);
  return cudaGetLastError();
}

template <typename T, bool UNI>
cudaError_t launch_phase_b(const Maps<SlotsB<T, UNI>::NH, SlotsB<T, UNI>::NC>& m, const Geom& g, T wc, T* t, double* part,
                           BicgState* st, const Launch& L) {
  typename OpB<T, UNI>::Args a{part, st, t, wc};
  return launch_stencil<OpB<T, UNI>>(m, a, g, L);
}

template <typename T, bool UNI>
cudaError_t launch_phase_ca(const Maps<SlotsCA<T, UNI>::NH, SlotsCA<T, UNI>::NC>& m, const Geom& g, T wc, T* x, T* r_out,
                            T* p_out, T* v_out, double* part, BicgState* st, int prime, const Launch& L) {
  typename OpCA<T, UNI>::Args a{part, st, x, r_out, p_out, v_out, wc, prime};
  return launch_stencil<OpCA<T, UNI>>(m, a, g, L);
}

template <typename T, bool UNI>
cudaError_t launch_cg_pass(const Maps<SlotsCG<T, UNI>::NH, SlotsCG<T, UNI>::NC>& m, const Geom& g, T wc, T* r_out,
                           T* w_out, T* s_out, T* p, T* x, double* part, BicgState* st, int prime, const Launch& L) {
  typename OpCG<T, UNI>::Args a{part, st, r_out, w_out, s_out, p, x, wc, prime};
  return launch_stencil<OpCG<T, UNI>>(m, a, g, L);
}

template <bool UNI>
cudaError_t launch_residual(const Maps<SlotsRes<UNI>::NH, SlotsRes<UNI>::NC>& m, const Geom& g, double wc,
                            double diagc, int init, double* r, double* rt, double* p, double* v, double* t, float* r32,
                            double* part, BicgState* st, const Launch& L, const ResidualExtras& ex) {
  typename OpRes<UNI>::Args a{part, st, wc, diagc, init, r, rt, p, v, t, r32};
  a.need_bb = ex.need_bb;
  a.need_max = ex.need_max;
  if (ex.st2) {
    a.in_r = ex.r;
    a.in_rt = ex.rt;
    a.in_p = ex.p;
    a.in_v = ex.v;
    a.in_t = ex.t;
    a.in_d = ex.d;
    a.st2 = ex.st2;
  }
  return launch_stencil<OpRes<UNI>>(m, a, g, L);
}

template <typename T>
cudaError_t launch_init_zero(const T* b, const Geom& g, T* r, T* rt, T* p, T* v, T* t, double* part, BicgState* st,
                             cudaStream_t s) {
  k_init_zero<T><<<row_blocks(g), NTHREADS, 0, s>>>(b, g, r, rt, p, v, t, part, st);
  return cudaGetLastError();
}

cudaError_t launch_add_f32(double* x, const float* d, long n, cudaStream_t s) {
  k_add_f32<<<ew_blocks(n), 256, 0, s>>>(x, d, n);
  return cudaGetLastError();
}

cudaError_t launch_set_state(BicgState* st, double tol, int norm, int max_iter, double tol_r0, int keep_r0,
                             cudaStream_t s) {
  k_set_state<<<1, 1, 0, s>>>(st, tol, norm, max_iter, tol_r0, keep_r0);
  return cudaGetLastError();
}

__global__ void k_mark_done(BicgState* st) { st->done = 1; }

// Self-test of the bounded wait that guards every TMA stage: one thread waits on an mbarrier on which
// nothing ever arrives; the wait must give up after `limit` cycles and report PF_E_TIMEOUT (7).
__global__ void k_wait_probe(unsigned long long limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) *status = mbar_wait(&bar, 0u, limit) ? 0 : 7;
}

cudaError_t launch_wait_probe(unsigned long long limit, int* status, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(limit, status);
  return cudaGetLastError();
}

cudaError_t launch_mark_done(BicgState* st, cudaStream_t s) {
  k_mark_done<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_plane_bb(const double* b, const Geom& g, double* part, BicgState* st, cudaStream_t s) {
  const int rows = 2 * g.ny;
  k_plane_bb<<<rows < 128 ? rows : 128, NTHREADS, 0, s>>>(b, g, part, st);
  return cudaGetLastError();
}

cudaError_t launch_faces(const double* eps, const Geom& g, double h, double* wE, double* wN, double* wU, double* dsum,
                         float* gh32, cudaStream_t s) {
  k_faces<<<row_blocks(g), 128, 0, s>>>(eps, g, 1.0 / (h * h), wE, wN, wU, dsum, gh32);
  return cudaGetLastError();
}

cudaError_t launch_spread(const double* charges, int nq, double ox, double oy, double oz, double h, double lam,
                          const Geom& g, double* f, int* err, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  k_spread<<<1, 32, 0, s>>>(charges, nq, ox, oy, oz, h, lam, g, f, err);
  return cudaGetLastError();
}

cudaError_t launch_eps_diag(const double* dsum, const double* sig, const uint8_t* smask, const Geom& g, double* diag,
                            double* dinv, float* dinv32, cudaStream_t s) {
  k_eps_diag<<<row_blocks(g), 128, 0, s>>>(dsum, sig, smask, g, diag, dinv, dinv32);
  return cudaGetLastError();
}

cudaError_t launch_pf1_dinv(const uint8_t* solvent, const Geom& g, double dinvc, double* dinv, float* dinv32,
                            cudaStream_t s) {
  k_pf1_dinv<<<row_blocks(g), 128, 0, s>>>(solvent, g, dinvc, dinv, dinv32);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* a, float* b, long n, cudaStream_t s) {
  k_to_f32<<<ew_blocks(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_impose(double* x, const double* b, const double* dinv, long n, cudaStream_t s) {
  k_impose<<<ew_blocks(n), 256, 0, s>>>(x, b, dinv, n);
  return cudaGetLastError();
}

cudaError_t launch_pack(const void* src, void* dst, const Geom& g, int type, cudaStream_t s) {
  if (type == 0)
    k_pack_d<<<row_blocks(g), 128, 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst), g);
  else
    k_pack_u8<<<row_blocks(g), 128, 0, s>>>(static_cast<const uint8_t*>(src), static_cast<uint8_t*>(dst), g);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const double* src, double* dst, const Geom& g, int count, cudaStream_t s) {
  k_unpack<<<row_blocks(g), 128, 0, s>>>(src, dst, g, count);
  return cudaGetLastError();
}

cudaError_t launch_fermi(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesParams& sp,
                         const Geom& g, double* b1, double* sig, double* c2, double* C, double* S, double* G,
                         double* ulast, int warm, int* err, cudaStream_t s, const float* u32start) {
  k_fermi<<<ew_blocks(g.np), 256, 0, s>>>(phi0, solvent, ffix, sp, g, b1, sig, c2, C, S, G, ulast, warm, err,
                                          u32start);
  return cudaGetLastError();
}

cudaError_t launch_fermi_df(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesDF& sp,
                            const Geom& g, double* b1, double* sig, double* c2, float* u32, int warm, int* err,
                            cudaStream_t s) {
  static const Exp2Table tab = make_exp2_table();
  k_fermi_df<<<ew_blocks(g.np), 256, 0, s>>>(phi0, solvent, ffix, sp, tab, g, b1, sig, c2, u32, warm, err);
  return cudaGetLastError();
}

cudaError_t launch_pf2_rhs(const double* psi, const uint8_t* solvent, const double* c2, double eps_s, double lo,
                           double hi, const Geom& g, double* b2, cudaStream_t s) {
  k_pf2_rhs<<<row_blocks(g), 128, 0, s>>>(psi, solvent, c2, eps_s, lo, hi, g, b2);
  return cudaGetLastError();
}

cudaError_t launch_relax(double* phi0, const double* phi, double omega, long n, double* part, unsigned int* ticket,
                         double* delta, cudaStream_t s) {
  k_relax<<<ew_blocks(n), NTHREADS, 0, s>>>(phi0, phi, omega, n, part, ticket, delta);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* a, double sc, double* out, long n, cudaStream_t s) {
  k_scale<<<ew_blocks(n), 256, 0, s>>>(a, sc, out, n);
  return cudaGetLastError();
}

cudaError_t launch_set_dirichlet(double* x, double lo, double hi, const Geom& g, cudaStream_t s) {
  k_set_dirichlet<<<row_blocks(g), 128, 0, s>>>(x, lo, hi, g);
  return cudaGetLastError();
}

// explicit instantiations
#define PF_INST(T, U)                                                                                               \
  template cudaError_t launch_phase_b<T, U>(const Maps<SlotsB<T, U>::NH, SlotsB<T, U>::NC>&, const Geom&, T, T*,   \
                                            double*, BicgState*, const Launch&);                                   \
  template cudaError_t launch_phase_ca<T, U>(const Maps<SlotsCA<T, U>::NH, SlotsCA<T, U>::NC>&, const Geom&, T, T*, \
                                             T*, T*, T*, double*, BicgState*, int, const Launch&);                 \
  template cudaError_t launch_cg_pass<T, U>(const Maps<SlotsCG<T, U>::NH, SlotsCG<T, U>::NC>&, const Geom&, T, T*,   \
                                            T*, T*, T*, T*, double*, BicgState*, int, const Launch&);
PF_INST(double, false)
PF_INST(double, true)
PF_INST(float, false)
PF_INST(float, true)
template cudaError_t launch_residual<false>(const Maps<SlotsRes<false>::NH, SlotsRes<false>::NC>&, const Geom&, double,
                                            double, int, double*, double*, double*, double*, double*, float*, double*,
                                            BicgState*, const Launch&, const ResidualExtras&);
template cudaError_t launch_residual<true>(const Maps<SlotsRes<true>::NH, SlotsRes<true>::NC>&, const Geom&, double,
                                           double, int, double*, double*, double*, double*, double*, float*, double*,
                                           BicgState*, const Launch&, const ResidualExtras&);
template cudaError_t launch_init_zero<float>(const float*, const Geom&, float*, float*, float*, float*, float*, double*,
                                             BicgState*, cudaStream_t);
template cudaError_t launch_init_zero<double>(const double*, const Geom&, double*, double*, double*, double*, double*,
                                              double*, BicgState*, cudaStream_t);

}  // namespace pf

// ====================================================================================================
// Entry point that allocates nothing: the pointwise Fermi/steric step on caller arrays.
//
// Some callers cannot allocate device memory at the moment they need this step: a host application
// that hands the library a fixed device arena, or code that runs where cudaMalloc is not allowed or
// would stall (a memory pool owned by another runtime, a latency-critical loop).  This variant of
// k_fermi keeps its scratch -- each node's ln Gamma, the warm start of the next call, and the
// root-failure flag -- in a file-scope device array of fixed size instead of in a pf_grid, so a call
// needs only the caller's input and output arrays.  The paper has no counterpart: it is a property of
// this library's interface only.
// ====================================================================================================
#include <mutex>

void pf_internal_set_error(const char* msg);  // pf_api.cu: the message pf_last_error returns

namespace pf {

// scratch: PF_FERMI_NOALLOC_MAX_NODES doubles of ln Gamma, then the failure flag (one 8-byte word)
static __device__ __align__(256) double g_fermi_scratch[PF_FERMI_NOALLOC_MAX_NODES + 1];

// Same arithmetic as k_fermi: phi arrives in volts (phi_hat = phi * inv_tv), C leaves in mol/L; arrays are
// compact (x fastest, n entries per field).  Like k_fermi's ulast, the scratch holds each solvent node's
// ln Gamma: read as the Newton start when warm != 0 (fermi_point clamps any start into its bracket, so
// stale or foreign contents only cost iterations), rewritten with the new root.
__global__ void k_fermi_noalloc(const double* __restrict__ phi_V, const uint8_t* __restrict__ solvent, long n,
                                SpeciesParams sp, double inv_tv, double inv_molar, int warm, double* C, double* S,
                                double* G, double* scratch) {
  double* ulast = scratch;
  unsigned long long* flag = reinterpret_cast<unsigned long long*>(scratch + PF_FERMI_NOALLOC_MAX_NODES);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double ph = phi_V[c] * inv_tv;
    const bool sol = solvent[c] != 0;
    FermiOut fo;
    bool ok = false;
    if (sol) {
      ok = fermi_point(sp, ph, warm ? ulast[c] : sp.lgB, fo);
      if (!ok) atomicExch(flag, 1ull);
      else ulast[c] = fo.u;
    }
    for (int s = 0; s < sp.ns; ++s) C[s * n + c] = (sol && ok) ? fo.C[s] * inv_molar : 0.0;
    if (S) S[c] = (sol && ok) ? fo.S : 0.0;
    if (G) G[c] = (sol && ok) ? fo.G : 0.0;
  }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

pf_status noalloc_fail(pf_status s, const char* msg) {
  pf_internal_set_error(msg);
  return s;
}
}  // namespace

}  // namespace pf

extern "C" {

pf_status pf_fermi_noalloc(long n, const double* phi_V, const uint8_t* solvent, int n_species,
                           const pf_species* species, double T_K, int warm_start, double* C_M, double* S,
                           double* Gamma, void* cuda_stream) {
  using namespace pf;
  if (n < 1 || n > PF_FERMI_NOALLOC_MAX_NODES)
    return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: n must be between 1 and PF_FERMI_NOALLOC_MAX_NODES");
  if (!phi_V || !solvent || !C_M || (warm_start != 0 && warm_start != 1))
    return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: phi_V, solvent and C_M are required, warm_start is 0 or 1");
  SpeciesParams sp{};
  double tv = 0.0, molar = 0.0;
  if (const char* why = species_params(n_species, species, T_K, &sp, &tv, &molar)) {
    static thread_local char msg[160];
    snprintf(msg, sizeof msg, "pf_fermi_noalloc: %s", why);
    return noalloc_fail(PF_E_INVAL, msg);
  }

  // set-up, once per device and with that device current: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: no current CUDA device");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_fermi_scratch);
      if (e != cudaSuccess || !p) return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: cudaGetSymbolAddress failed");
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the failure flag must start at zero; the ln Gamma part is only a starting point (read when warm_start)
  if (cudaMemsetAsync(scratch + PF_FERMI_NOALLOC_MAX_NODES, 0, sizeof(double), s) != cudaSuccess)
    return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: clearing the flag failed");
  long blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_fermi_noalloc<<<(int)blocks, 256, 0, s>>>(phi_V, solvent, n, sp, 1.0 / tv, 1.0 / molar, warm_start, C_M, S,
                                              Gamma, scratch);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: launch failed");
  unsigned long long flag = 0;
  if (cudaMemcpyAsync(&flag, scratch + PF_FERMI_NOALLOC_MAX_NODES, sizeof(flag), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: kernel failed");
  if (flag) return noalloc_fail(PF_E_GAMMA, "pf_fermi_noalloc: the void-fraction root was not found");
  return PF_OK;
}

}  // extern "C"

namespace pf {

// ------------------------------------------------------------------ Anderson acceleration of the outer loop
// f = g - x at the new outer iterate (g: the PF2 solution from x), the newest history columns
// dF = f - f_prev and dX = x - x_prev (when have_prev), then f_prev <- f, x_prev <- x; the block maxima of
// |f| go to part, the last block writes max |f| to *fmax.
__global__ void __launch_bounds__(NTHREADS) k_aa_residual(const double* __restrict__ gval, const double* __restrict__ x,
                                                          double* __restrict__ f, double* __restrict__ fprev,
                                                          double* __restrict__ xprev, double* __restrict__ dF,
                                                          double* __restrict__ dX, int have_prev, long n,
                                                          double* part, unsigned int* ticket, double* fmax_out) {
  __shared__ double scratch[NTHREADS];
  double m = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double xc = x[c], fc = gval[c] - xc;
    if (have_prev) {
      dF[c] = fc - fprev[c];
      dX[c] = xc - xprev[c];
    }
    f[c] = fc;
    fprev[c] = fc;
    xprev[c] = xc;
    m = fmax(m, fabs(fc));
  }
  double vals[1] = {m};
  block_partials<1>(vals, 1u, part, scratch);
  if (!arrive_last(ticket)) return;
  double tot[1];
  total_partials<1>(part, 1u, tot, scratch);
  if (threadIdx.x == 0) {
    *fmax_out = tot[0];
    *ticket = 0;
  }
}

// Inner products of the Anderson least-squares problem: out[j] = dF_new . dF_j and out[AA_MAX + j] = dF_j . f
// for the k active columns.
__global__ void __launch_bounds__(NTHREADS) k_aa_dots(AAPtrs cols, int k, const double* __restrict__ dFnew,
                                                      const double* __restrict__ f, long n, double* part,
                                                      unsigned int* ticket, double* out) {
  __shared__ double scratch[NTHREADS * 2 * AA_MAX];
  double a[2 * AA_MAX];
#pragma unroll
  for (int j = 0; j < 2 * AA_MAX; ++j) a[j] = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double dn = dFnew[c], fc = f[c];
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j) {
      if (j < k) {
        const double d = cols.dF[j][c];
        a[j] = fma(dn, d, a[j]);
        a[AA_MAX + j] = fma(d, fc, a[AA_MAX + j]);
      }
    }
  }
  // the block partial vectors are reduced with the same fixed-order machinery as the solver's dots
  block_partials<2 * AA_MAX>(a, 0u, part, scratch);
  if (!arrive_last(ticket)) return;
  double tot[2 * AA_MAX];
  total_partials<2 * AA_MAX>(part, 0u, tot, scratch);
  if (threadIdx.x == 0) {
    for (int j = 0; j < 2 * AA_MAX; ++j) out[j] = tot[j];
    *ticket = 0;
  }
}

// x <- x + beta f - sum_j gamma_j (dX_j + beta dF_j) over the k active columns.
__global__ void k_aa_update(AAPtrs cols, AACoef gam, int k, double beta, double* __restrict__ x,
                            const double* __restrict__ f, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    double v = fma(beta, f[c], x[c]);
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j)
      if (j < k) v -= gam.g[j] * fma(beta, cols.dF[j][c], cols.dX[j][c]);
    x[c] = v;
  }
}

cudaError_t launch_aa_residual(const double* gval, const double* x, double* f, double* fprev, double* xprev,
                               double* dF, double* dX, int have_prev, long n, double* part, unsigned int* ticket,
                               double* fmax_out, cudaStream_t s) {
  k_aa_residual<<<ew_blocks(n), NTHREADS, 0, s>>>(gval, x, f, fprev, xprev, dF, dX, have_prev, n, part, ticket,
                                                  fmax_out);
  return cudaGetLastError();
}

cudaError_t launch_aa_dots(const AAPtrs& cols, int k, const double* dFnew, const double* f, long n, double* part,
                           unsigned int* ticket, double* out, cudaStream_t s) {
  k_aa_dots<<<ew_blocks(n), NTHREADS, 0, s>>>(cols, k, dFnew, f, n, part, ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_aa_update(const AAPtrs& cols, const AACoef& gam, int k, double beta, double* x, const double* f,
                             long n, cudaStream_t s) {
  k_aa_update<<<ew_blocks(n), 256, 0, s>>>(cols, gam, k, beta, x, f, n);
  return cudaGetLastError();
}

}  // namespace pf
