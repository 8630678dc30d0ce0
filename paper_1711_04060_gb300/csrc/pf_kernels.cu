// pf_kernels.cu -- sm_103a kernels of the Poisson-Fermi hot path.
//
// Stencil kernels walk 2D tiles (TX x TY nodes in x-y, one warp per x row, so every global
// access of a warp is one coalesced row segment) up through a chunk of ZC interior z-planes.
// The stencil input of a plane is computed once per node (with its one-node x-y halo) into a
// shared-memory plane; the planes below and above come from registers of the same thread, so a
// node's input vectors are read from DRAM once per kernel (halo rows of neighbouring tiles come
// from L2).  The axpy updates of BiCGSTAB (Table 3 steps 9, 13, 16, 17), the Jacobi scaling
// and the inner products (steps 4, 12, 15) are fused into the two stencil kernels of an
// iteration; each kernel's inner products are reduced by warp shuffles, a block tree and a
// last-arriving-block pass over the per-block partials in fixed order (deterministic).
#include <math.h>

#include "pf_internal.cuh"

namespace pf {

// ------------------------------------------------------------------ accumulation helpers
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// FP32 products summed with an error-free transformation (TwoProduct by FMA, TwoSum), so a
// thread's partial sum carries about twice the FP32 precision before it is handed to the
// FP64 block reduction.
template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float t = __fadd_rn(hi, p);
    const float z = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
__device__ __forceinline__ T tabs(T a) { return a < T(0) ? -a : a; }

// Reduce NV per-thread values over the block (value j is a max when bit j of maxmask is set,
// else a sum) and store the block's result in part[blockIdx.x * NPART + j].
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], unsigned maxmask, double* part) {
  __shared__ double red[NTHREADS / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double a = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_down_sync(0xffffffffu, a, o);
      a = ((maxmask >> j) & 1u) ? fmax(a, b) : a + b;
    }
    if (lane == 0) red[warp][j] = a;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double a = red[0][j];
    for (int w = 1; w < NTHREADS / 32; ++w) a = ((maxmask >> j) & 1u) ? fmax(a, red[w][j]) : a + red[w][j];
    part[blockIdx.x * NPART + j] = a;
  }
}

// Returns true in the block that arrives last; that block then sees every partial.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: totals over all blocks' partials, in fixed order.
template <int NV>
__device__ __forceinline__ void total_partials(const double* part, unsigned maxmask, double (&tot)[NV]) {
  __shared__ double red[NTHREADS][NV];
  double a[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) a[j] = 0.0;  // sums start at 0; maxima are of absolute values
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NTHREADS) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const double x = __ldcg(part + (long)b * NPART + j);
      a[j] = ((maxmask >> j) & 1u) ? fmax(a[j], x) : a[j] + x;
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) red[threadIdx.x][j] = a[j];
  __syncthreads();
  for (int s = NTHREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int j = 0; j < NV; ++j)
        red[threadIdx.x][j] = ((maxmask >> j) & 1u) ? fmax(red[threadIdx.x][j], red[threadIdx.x + s][j])
                                                     : red[threadIdx.x][j] + red[threadIdx.x + s][j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = red[0][j];
}

// ------------------------------------------------------------------ tile geometry
int tiles_for(int nx, int ny, int nz) {
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, nzc = (nz - 2 + ZC - 1) / ZC;
  return ntx * nty * nzc;
}

struct Tile {
  int x0, y0, kb, ke;
};

__device__ __forceinline__ Tile tile_of(int t, int nx, int ny, int nz) {
  const int nzc = (nz - 2 + ZC - 1) / ZC, ntx = (nx + TX - 1) / TX;
  const int zc = t % nzc, xy = t / nzc;
  Tile r;
  r.x0 = (xy % ntx) * TX;
  r.y0 = (xy / ntx) * TY;
  r.kb = 1 + zc * ZC;
  r.ke = min(r.kb + ZC, nz - 1);
  return r;
}

// Position g in [-1, n] of a tile (with halo) -> node index whose value it holds: the node
// itself, the mirror image for the two ghost positions (zero-flux sides, Eq. 4), or -1 when
// no output of the tile uses it.
__device__ __forceinline__ int mirror(int g, int n) {
  if (g < 0) return 1;
  if (g < n) return g;
  if (g == n) return n - 2;
  return -1;
}

constexpr int PW = TX + 2;                 // smem plane row pitch
constexpr int PLANE = (TY + 2) * PW;       // smem plane size
constexpr int NHALO = 2 * (TX + 2) + 2 * TY;

// halo slot h (0..NHALO-1) -> tile-local (lx, ly) in [-1, TX] x [-1, TY]
__device__ __forceinline__ void halo_pos(int h, int& lx, int& ly) {
  if (h < TX + 2) { lx = h - 1; ly = -1; return; }
  h -= TX + 2;
  if (h < TX + 2) { lx = h - 1; ly = TY; return; }
  h -= TX + 2;
  if (h < TY) { lx = -1; ly = h; return; }
  h -= TY;
  lx = TX;
  ly = h;
}

// Per-thread geometry of one tile: the (mirrored) x-y offsets of the thread's centre and halo slot.
struct TileGeo {
  long cxy;       // x-y offset of the centre position (or -1)
  long hxy;       // x-y offset of the halo slot (or -1 / no slot)
  int hs;         // smem index of the halo slot
  int gi, gj;     // centre node
  bool valid;     // centre is a real node (produces output)
};

__device__ __forceinline__ TileGeo tile_geo(const Tile& tl, int nx, int ny) {
  TileGeo g;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  g.gi = tl.x0 + lx;
  g.gj = tl.y0 + ly;
  g.valid = g.gi < nx && g.gj < ny;
  const int mi = mirror(g.gi, nx), mj = mirror(g.gj, ny);
  g.cxy = (mi >= 0 && mj >= 0) ? (mi + (long)nx * mj) : -1;
  g.hxy = -1;
  g.hs = -1;
  if (threadIdx.x < NHALO) {
    int hx, hy;
    halo_pos(threadIdx.x, hx, hy);
    const int hi = mirror(tl.x0 + hx, nx), hj = mirror(tl.y0 + hy, ny);
    g.hs = (hy + 1) * PW + (hx + 1);
    g.hxy = (hi >= 0 && hj >= 0) ? (hi + (long)nx * hj) : -1;
  }
  return g;
}

__device__ __forceinline__ int cs(int lx, int ly) { return (ly + 1) * PW + (lx + 1); }

// Weighted neighbour sum of the 7-point operator at an output node: sum_nb w_nb q_nb with the
// west/south faces taken from the neighbour's east/north face (or the node's own at a mirror
// side) and the down face carried from the plane below.
template <typename T, bool UNI>
__device__ __forceinline__ T nb_sum(const OpView<T>& op, const T* cur, int lx, int ly, long c, int gi, int gj,
                                    T q_up, T q_dn, T wU_c, T wD) {
  const T qE = cur[cs(lx + 1, ly)], qW = cur[cs(lx - 1, ly)];
  const T qN = cur[cs(lx, ly + 1)], qS = cur[cs(lx, ly - 1)];
  if (UNI) {
    return op.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
  } else {
    const T wE = __ldg(op.wE + c), wW = __ldg(op.wE + c - (gi > 0 ? 1 : 0));
    const T wN = __ldg(op.wN + c), wS = __ldg(op.wN + c - (gj > 0 ? op.nx : 0));
    T a = wE * qE;
    a = fma(wW, qW, a);
    a = fma(wN, qN, a);
    a = fma(wS, qS, a);
    a = fma(wU_c, q_up, a);
    a = fma(wD, q_dn, a);
    return a;
  }
}

template <typename T, bool UNI>
__device__ __forceinline__ T face_up(const OpView<T>& op, long c) {
  if (UNI) return op.wc;
  return __ldg(op.wU + c);
}

// ------------------------------------------------------------------ BiCGSTAB init
// r = b - A x (x already holds b on identity rows), r~ = r, p = v = t = 0; partials: b.b, r.r, max|r|.
template <typename T, bool UNI>
__global__ void __launch_bounds__(NTHREADS) k_init(OpView<T> op, const T* __restrict__ x, int x_zero,
                                                   const T* __restrict__ b, T* __restrict__ r, T* __restrict__ rt,
                                                   T* __restrict__ p, T* __restrict__ v, T* __restrict__ t,
                                                   double* part, BicgState* st, int ntiles) {
  __shared__ T Qa[PLANE], Qb[PLANE];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long sxy = (long)nx * ny;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  Acc<T> abb, arr;
  T rmax = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tl = tile_of(tile, nx, ny, nz);
    const TileGeo g = tile_geo(tl, nx, ny);
    T* cur = Qa;
    T* nxt = Qb;
    auto xq = [&](long id) -> T { return x_zero ? T(0) : x[id]; };
    T q_dn = (g.cxy >= 0) ? xq(g.cxy + (tl.kb - 1) * sxy) : T(0);
    T q_c = (g.cxy >= 0) ? xq(g.cxy + tl.kb * sxy) : T(0);
    cur[cs(lx, ly)] = q_c;
    if (g.hs >= 0) cur[g.hs] = (g.hxy >= 0) ? xq(g.hxy + tl.kb * sxy) : T(0);
    T wD = (g.cxy >= 0 && !x_zero) ? face_up<T, UNI>(op, g.cxy + (tl.kb - 1) * sxy) : T(0);
    __syncthreads();
    for (int k = tl.kb; k < tl.ke; ++k) {
      const T q_up = (g.cxy >= 0) ? xq(g.cxy + (k + 1) * sxy) : T(0);
      nxt[cs(lx, ly)] = q_up;
      if (g.hs >= 0) nxt[g.hs] = (g.hxy >= 0) ? xq(g.hxy + (k + 1) * sxy) : T(0);
      __syncthreads();
      if (g.valid) {
        const long c = g.gi + (long)nx * g.gj + k * sxy;
        const T bc = b[c];
        T rc;
        T wU_c = T(0);
        if (x_zero) {
          rc = bc;
        } else {
          wU_c = face_up<T, UNI>(op, c);
          const T dv = op.dinv[c];
          if (dv == T(0)) {
            rc = bc - q_c;
          } else {
            const T diag = UNI ? T(op.diagc) : (op.diag ? T(op.diag[c]) : T(1) / dv);
            const T a = nb_sum<T, UNI>(op, cur, lx, ly, c, g.gi, g.gj, q_up, q_dn, wU_c, wD);
            rc = bc - (diag * q_c - a);
          }
        }
        r[c] = rc;
        rt[c] = rc;
        p[c] = T(0);
        v[c] = T(0);
        t[c] = T(0);
        abb.prod(bc, bc);
        arr.prod(rc, rc);
        rmax = fmax(rmax, tabs(rc));
        wD = wU_c;
      }
      __syncthreads();
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
      q_dn = q_c;
      q_c = q_up;
    }
    __syncthreads();
  }
  double vals[3] = {abb.value(), arr.value(), (double)rmax};
  block_partials<3>(vals, 4u, part);
  if (arrive_last(&st->ticket)) {
    double tot[3];
    total_partials<3>(part, 4u, tot);
    if (threadIdx.x == 0) {
      // Dirichlet planes: r = b - x = 0 there, b may be nonzero; the norms above skip them, so add b.b of
      // the planes through the host (st->bnorm2 is preset to that value).
      double bb = tot[0] + st->bnorm2;
      if (bb == 0.0) bb = 1.0;
      st->bnorm2 = bb;
      st->rho = tot[1];
      st->rnorm2 = tot[1];
      st->rinf = tot[2];
      st->tol2 = st->tol * st->tol * bb;
      st->alpha = st->omega = st->beta = 0.0;
      st->sexit = 0;
      st->iter = 0;
      const bool conv = st->norm == 0 ? (tot[1] <= st->tol2) : (tot[2] < st->tol);
      st->done = conv ? 1 : 0;
      st->status = 0;
      st->ticket = 0;
    }
  }
}

// ------------------------------------------------------------------ BiCGSTAB phase B
// s = r - alpha v (step 13), t = A M^-1 s (step 14); partials r~.s, r~.t, t.s, t.t, s.s, max|s|.
template <typename T, bool UNI>
__global__ void __launch_bounds__(NTHREADS) k_phase_b(OpView<T> op, const T* __restrict__ r,
                                                      const T* __restrict__ v, const T* __restrict__ rt,
                                                      T* __restrict__ t, double* part, BicgState* st, int ntiles) {
  if (*(volatile int*)&st->done) return;
  __shared__ T Qa[PLANE], Qb[PLANE];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long sxy = (long)nx * ny;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const T al = (T)st->alpha;
  Acc<T> a_rs, a_rt, a_ts, a_tt, a_ss;
  T smax = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tl = tile_of(tile, nx, ny, nz);
    const TileGeo g = tile_geo(tl, nx, ny);
    T* cur = Qa;
    T* nxt = Qb;
    auto sq = [&](long id, T& s_) -> T {
      s_ = fma(-al, v[id], r[id]);
      return op.dinv[id] * s_;
    };
    T s_dn, s_c, s_up;
    T q_dn = (g.cxy >= 0) ? sq(g.cxy + (tl.kb - 1) * sxy, s_dn) : T(0);
    T q_c = T(0);
    s_c = T(0);
    if (g.cxy >= 0) q_c = sq(g.cxy + tl.kb * sxy, s_c);
    cur[cs(lx, ly)] = q_c;
    if (g.hs >= 0) {
      T dummy;
      cur[g.hs] = (g.hxy >= 0) ? sq(g.hxy + tl.kb * sxy, dummy) : T(0);
    }
    T wD = (g.cxy >= 0) ? face_up<T, UNI>(op, g.cxy + (tl.kb - 1) * sxy) : T(0);
    __syncthreads();
    for (int k = tl.kb; k < tl.ke; ++k) {
      T q_up = T(0);
      s_up = T(0);
      if (g.cxy >= 0) q_up = sq(g.cxy + (k + 1) * sxy, s_up);
      nxt[cs(lx, ly)] = q_up;
      if (g.hs >= 0) {
        T dummy;
        nxt[g.hs] = (g.hxy >= 0) ? sq(g.hxy + (k + 1) * sxy, dummy) : T(0);
      }
      __syncthreads();
      if (g.valid) {
        const long c = g.gi + (long)nx * g.gj + k * sxy;
        const T wU_c = face_up<T, UNI>(op, c);
        T tc;
        if (op.dinv[c] == T(0)) {
          tc = s_c;
        } else {
          tc = s_c - nb_sum<T, UNI>(op, cur, lx, ly, c, g.gi, g.gj, q_up, q_dn, wU_c, wD);
        }
        t[c] = tc;
        const T rtc = rt[c];
        a_rs.prod(rtc, s_c);
        a_rt.prod(rtc, tc);
        a_ts.prod(tc, s_c);
        a_tt.prod(tc, tc);
        a_ss.prod(s_c, s_c);
        smax = fmax(smax, tabs(s_c));
        wD = wU_c;
      }
      __syncthreads();
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
      q_dn = q_c;
      q_c = q_up;
      s_c = s_up;
    }
    __syncthreads();
  }
  double vals[6] = {a_rs.value(), a_rt.value(), a_ts.value(), a_tt.value(), a_ss.value(), (double)smax};
  block_partials<6>(vals, 32u, part);
  if (arrive_last(&st->ticket)) {
    double tot[6];
    total_partials<6>(part, 32u, tot);
    if (threadIdx.x == 0) {
      const double rs = tot[0], rtt = tot[1], ts = tot[2], tt = tot[3], ss = tot[4], smx = tot[5];
      st->snorm2 = ss;
      st->sinf = smx;
      const bool sconv = st->norm == 0 ? (ss <= st->tol2) : (smx < st->tol);
      if (sconv) {  // early exit of the Templates algorithm: x += alpha M^-1 p, r = s
        st->sexit = 1;
        st->omega = 0.0;
        st->beta = 0.0;
      } else if (tt == 0.0 || !isfinite(tt) || !isfinite(ts) || !isfinite(ss)) {
        st->status = 4;  // PF_E_BREAKDOWN (a zero or non-finite t.t stops before x is touched)
        st->done = 1;
      } else {
        const double om = ts / tt;  // step 15
        st->omega = om;
        // r~.r_new with r_new = s - omega t (steps 17 and 4 of the next iteration), needed now
        // because the next p is formed in the same kernel as r_new
        const double rho_new = rs - om * rtt;
        const double be = (om != 0.0) ? (rho_new / st->rho) * (st->alpha / om) : 0.0;  // step 8
        st->beta = isfinite(be) ? be : 0.0;
      }
      st->ticket = 0;
    }
  }
}

// ------------------------------------------------------------------ BiCGSTAB phase C+A
// s = r - alpha v, x += alpha M^-1 p + omega M^-1 s (step 16), r' = s - omega t (step 17),
// p' = r' + beta (p - omega v) (step 9 of the next iteration), v' = A M^-1 p' (step 11);
// partials r~.v', r~.r', r'.r', max|r'|.  With prime = 1 (alpha = omega = beta = 0) it forms the
// first p = r0 and v = A M^-1 r0.
template <typename T, bool UNI>
__global__ void __launch_bounds__(NTHREADS) k_phase_ca(OpView<T> op, const T* __restrict__ r,
                                                       const T* __restrict__ v, const T* __restrict__ p,
                                                       const T* __restrict__ t, const T* __restrict__ rt,
                                                       T* __restrict__ x, T* __restrict__ r_out,
                                                       T* __restrict__ p_out, T* __restrict__ v_out, double* part,
                                                       BicgState* st, int prime, int ntiles) {
  if (*(volatile int*)&st->done) return;
  __shared__ T Qa[PLANE], Qb[PLANE];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long sxy = (long)nx * ny;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const T al = (T)st->alpha, om = (T)st->omega, be = (T)st->beta;
  Acc<T> a_rv, a_rr, a_r2;
  T rmax = 0;
  struct Ctr {
    T s, rn, pn, pold, di;
  };
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tl = tile_of(tile, nx, ny, nz);
    const TileGeo g = tile_geo(tl, nx, ny);
    T* cur = Qa;
    T* nxt = Qb;
    auto pq = [&](long id, Ctr& o) -> T {
      const T vv = v[id], pp = p[id];
      o.s = fma(-al, vv, r[id]);
      o.rn = fma(-om, t[id], o.s);
      o.pn = fma(be, fma(-om, vv, pp), o.rn);
      o.pold = pp;
      o.di = op.dinv[id];
      return o.di * o.pn;
    };
    Ctr cd, cc, cu;
    T q_dn = (g.cxy >= 0) ? pq(g.cxy + (tl.kb - 1) * sxy, cd) : T(0);
    T q_c = T(0);
    cc.s = cc.rn = cc.pn = cc.pold = cc.di = T(0);
    if (g.cxy >= 0) q_c = pq(g.cxy + tl.kb * sxy, cc);
    cur[cs(lx, ly)] = q_c;
    if (g.hs >= 0) {
      Ctr dummy;
      cur[g.hs] = (g.hxy >= 0) ? pq(g.hxy + tl.kb * sxy, dummy) : T(0);
    }
    T wD = (g.cxy >= 0) ? face_up<T, UNI>(op, g.cxy + (tl.kb - 1) * sxy) : T(0);
    __syncthreads();
    for (int k = tl.kb; k < tl.ke; ++k) {
      T q_up = T(0);
      cu.s = cu.rn = cu.pn = cu.pold = cu.di = T(0);
      if (g.cxy >= 0) q_up = pq(g.cxy + (k + 1) * sxy, cu);
      nxt[cs(lx, ly)] = q_up;
      if (g.hs >= 0) {
        Ctr dummy;
        nxt[g.hs] = (g.hxy >= 0) ? pq(g.hxy + (k + 1) * sxy, dummy) : T(0);
      }
      __syncthreads();
      if (g.valid) {
        const long c = g.gi + (long)nx * g.gj + k * sxy;
        const T wU_c = face_up<T, UNI>(op, c);
        T vn;
        if (cc.di == T(0)) {
          vn = cc.pn;
        } else {
          vn = cc.pn - nb_sum<T, UNI>(op, cur, lx, ly, c, g.gi, g.gj, q_up, q_dn, wU_c, wD);
          if (!prime) {
            T xc = x[c];
            xc = fma(al, cc.di * cc.pold, xc);
            xc = fma(om, cc.di * cc.s, xc);
            x[c] = xc;
          }
        }
        r_out[c] = cc.rn;
        p_out[c] = cc.pn;
        v_out[c] = vn;
        const T rtc = rt[c];
        a_rv.prod(rtc, vn);
        a_rr.prod(rtc, cc.rn);
        a_r2.prod(cc.rn, cc.rn);
        rmax = fmax(rmax, tabs(cc.rn));
        wD = wU_c;
      }
      __syncthreads();
      T* tmp = cur;
      cur = nxt;
      nxt = tmp;
      q_dn = q_c;
      q_c = q_up;
      cc = cu;
    }
    __syncthreads();
  }
  double vals[4] = {a_rv.value(), a_rr.value(), a_r2.value(), (double)rmax};
  block_partials<4>(vals, 8u, part);
  if (arrive_last(&st->ticket)) {
    double tot[4];
    total_partials<4>(part, 8u, tot);
    if (threadIdx.x == 0) {
      const double rv = tot[0], rr = tot[1], r2 = tot[2], rmx = tot[3];
      st->ticket = 0;
      if (!prime) {
        st->iter += 1;
        st->rnorm2 = r2;
        st->rinf = rmx;
        const bool conv = st->norm == 0 ? (r2 <= st->tol2) : (rmx < st->tol);
        if (st->sexit || conv) {
          st->done = 1;
          st->status = 0;
          return;
        }
        if (st->omega == 0.0) {
          st->done = 1;
          st->status = 4;
          return;
        }
        if (st->iter >= st->max_iter) {
          st->done = 1;
          st->status = 3;  // PF_E_NOCONV
          return;
        }
      }
      if (rr == 0.0 || rv == 0.0 || !isfinite(rr) || !isfinite(rv) || !isfinite(rr / rv)) {
        st->done = 1;
        st->status = 4;
        return;
      }
      st->rho = rr;        // step 4 of the next iteration
      st->alpha = rr / rv; // step 12 of the next iteration
    }
  }
}

// ------------------------------------------------------------------ FP64 residual (refinement)
// r = b - A x in FP64; writes r32 = rt32 = (float) r; partials r.r, max|r|, b.b.
template <bool UNI>
__global__ void __launch_bounds__(NTHREADS) k_residual(OpView<double> op, const double* __restrict__ x,
                                                       const double* __restrict__ b, float* __restrict__ r32,
                                                       double* part, BicgState* st, int ntiles) {
  __shared__ double Qa[PLANE], Qb[PLANE];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long sxy = (long)nx * ny;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  double arr = 0.0, abb = 0.0, rmax = 0.0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tl = tile_of(tile, nx, ny, nz);
    const TileGeo g = tile_geo(tl, nx, ny);
    double* cur = Qa;
    double* nxt = Qb;
    double q_dn = (g.cxy >= 0) ? x[g.cxy + (tl.kb - 1) * sxy] : 0.0;
    double q_c = (g.cxy >= 0) ? x[g.cxy + tl.kb * sxy] : 0.0;
    cur[cs(lx, ly)] = q_c;
    if (g.hs >= 0) cur[g.hs] = (g.hxy >= 0) ? x[g.hxy + tl.kb * sxy] : 0.0;
    double wD = (g.cxy >= 0) ? face_up<double, UNI>(op, g.cxy + (tl.kb - 1) * sxy) : 0.0;
    __syncthreads();
    for (int k = tl.kb; k < tl.ke; ++k) {
      const double q_up = (g.cxy >= 0) ? x[g.cxy + (k + 1) * sxy] : 0.0;
      nxt[cs(lx, ly)] = q_up;
      if (g.hs >= 0) nxt[g.hs] = (g.hxy >= 0) ? x[g.hxy + (k + 1) * sxy] : 0.0;
      __syncthreads();
      if (g.valid) {
        const long c = g.gi + (long)nx * g.gj + k * sxy;
        const double wU_c = face_up<double, UNI>(op, c);
        const double bc = b[c];
        double rc;
        if (op.dinv[c] == 0.0) {
          rc = bc - q_c;
        } else {
          const double diag = UNI ? op.diagc : op.diag[c];
          rc = bc - (diag * q_c - nb_sum<double, UNI>(op, cur, lx, ly, c, g.gi, g.gj, q_up, q_dn, wU_c, wD));
        }
        r32[c] = (float)rc;
        arr = fma(rc, rc, arr);
        abb = fma(bc, bc, abb);
        rmax = fmax(rmax, fabs(rc));
        wD = wU_c;
      }
      __syncthreads();
      double* tmp = cur;
      cur = nxt;
      nxt = tmp;
      q_dn = q_c;
      q_c = q_up;
    }
    __syncthreads();
  }
  double vals[3] = {arr, abb, rmax};
  block_partials<3>(vals, 4u, part);
  if (arrive_last(&st->ticket)) {
    double tot[3];
    total_partials<3>(part, 4u, tot);
    if (threadIdx.x == 0) {
      st->rnorm2 = tot[0];
      st->rinf = tot[2];
      double bb = tot[1] + st->bnorm2;  // bnorm2 preset to b.b over the Dirichlet planes
      if (bb == 0.0) bb = 1.0;
      st->bnorm2 = bb;
      st->tol2 = st->tol * st->tol * bb;
      st->done = (st->norm == 0 ? (tot[0] <= st->tol2) : (tot[2] < st->tol)) ? 1 : 0;
      st->ticket = 0;
    }
  }
}

// ------------------------------------------------------------------ setup kernels (a1)
__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

// Harmonic face coefficients (Eqs. 15-18 with zero jump) divided by h^2, stored per node for the
// east, north and up faces; at i = nx-1 (j = ny-1) the east (north) face is the mirror face to the
// ghost node.  dsum = sum of the six faces (the diagonal of -div(eps grad)), 1 on Dirichlet planes.
__global__ void k_faces(const double* __restrict__ eps, int nx, int ny, int nz, double ih2, double* wE,
                        double* wN, double* wU, double* dsum) {
  const long N = (long)nx * ny * nz, sxy = (long)nx * ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / sxy);
    const double e = eps[c];
    const double fe = __dmul_rn(harm(e, eps[i < nx - 1 ? c + 1 : c - 1]), ih2);
    const double fw = __dmul_rn(harm(e, eps[i > 0 ? c - 1 : c + 1]), ih2);
    const double fn = __dmul_rn(harm(e, eps[j < ny - 1 ? c + nx : c - nx]), ih2);
    const double fs = __dmul_rn(harm(e, eps[j > 0 ? c - nx : c + nx]), ih2);
    const double fu = k < nz - 1 ? __dmul_rn(harm(e, eps[c + sxy]), ih2) : 0.0;
    const double fd = k > 0 ? __dmul_rn(harm(e, eps[c - sxy]), ih2) : 0.0;
    wE[c] = fe;
    wN[c] = fn;
    wU[c] = fu;
    // same summation order as the assembled diagonal: east, west, north, south, up, down
    double d = __dadd_rn(fe, fw);
    d = __dadd_rn(d, fn);
    d = __dadd_rn(d, fs);
    d = __dadd_rn(d, fu);
    d = __dadd_rn(d, fd);
    dsum[c] = (k == 0 || k == nz - 1) ? 1.0 : d;
  }
}

// Trilinear spreading of the fixed charges (Eq. 3 on the grid): one thread, charges in order.
__global__ void k_spread(const double* __restrict__ ch, int nq, double ox, double oy, double oz, double h, double lam,
                         int nx, int ny, int nz, double* f, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double org[3] = {ox, oy, oz};
  const int n[3] = {nx, ny, nz};
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
      const long id = (i0[0] + dx) + (long)nx * ((i0[1] + dy) + (long)ny * (i0[2] + dz));
      f[id] = __dadd_rn(f[id], __dmul_rn(amp, w));
    }
  }
}

__global__ void k_eps_diag(const double* __restrict__ dsum, const double* __restrict__ sig,
                           const uint8_t* __restrict__ smask, int nx, int ny, int nz, double* diag, double* dinv,
                           float* dinv32) {
  const long N = (long)nx * ny * nz, sxy = (long)nx * ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const long k = c / sxy;
    double d = 1.0, di = 0.0;
    if (k > 0 && k < nz - 1) {
      d = dsum[c];
      if (sig && (!smask || smask[c])) d = __dadd_rn(d, sig[c]);
      di = 1.0 / d;
    }
    diag[c] = d;
    dinv[c] = di;
    if (dinv32) dinv32[c] = (float)di;
  }
}

__global__ void k_pf1_dinv(const uint8_t* __restrict__ solvent, int nx, int ny, int nz, double dinvc, double* dinv,
                           float* dinv32) {
  const long N = (long)nx * ny * nz, sxy = (long)nx * ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const long k = c / sxy;
    const double di = (k > 0 && k < nz - 1 && solvent[c]) ? dinvc : 0.0;
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

// ------------------------------------------------------------------ Eq. (1) pointwise step
// Void fraction Gamma = e^u from f(u) = e^u + sum_i exp(la_i + p_i u) - 1 = 0 (bracketed Newton in u),
// S = u - ln Gamma^B, C_i = cB_i exp(-z_i phi + p_i S), rho = sum z_i C_i, kappa = lambda sum z_i^2 C_i.
__device__ __forceinline__ bool fermi_root(const SpeciesParams& sp, double phi, double& u_out, double (&la)[MAXSP]) {
  int nterm = 0;
  for (int i = 0; i < sp.ns; ++i) {
    la[i] = sp.lvc[i] - sp.z[i] * phi - sp.p[i] * sp.lgB;
    if (sp.lvc[i] > -INFINITY) ++nterm;
  }
  const double lnn = log((double)(nterm + 1));
  double hi = 0.0, lo = -lnn;
  for (int i = 0; i < sp.ns; ++i) {
    if (!(sp.lvc[i] > -INFINITY)) continue;
    const double a = -la[i] / sp.p[i], b = (-la[i] - lnn) / sp.p[i];
    hi = fmin(hi, a);
    lo = fmin(lo, b);
  }
  double u = sp.lgB;
  if (!(u < hi && u > lo)) u = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    const double eu = exp(u);
    double f = eu - 1.0, df = eu;
    for (int i = 0; i < sp.ns; ++i) {
      if (!(sp.lvc[i] > -INFINITY)) continue;
      const double term = exp(la[i] + sp.p[i] * u);
      f += term;
      df += sp.p[i] * term;
    }
    if (f == 0.0) {
      u_out = u;
      return true;
    }
    if (f > 0.0) hi = u; else lo = u;
    double un = u - f / df;
    if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
    const double du = un - u;
    u = un;
    if (fabs(du) <= 1e-15 * fmax(1.0, fabs(u))) {
      u_out = u;
      return isfinite(u);
    }
  }
  return false;
}

__global__ void k_fermi(const double* __restrict__ phi0, const uint8_t* __restrict__ solvent,
                        const double* __restrict__ ffix, SpeciesParams sp, int nx, int ny, int nz, double* b1,
                        double* sig, double* c2, double* C, double* S, double* G, int* err) {
  const long N = (long)nx * ny * nz, sxy = (long)nx * ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const long k = c / sxy;
    const double ph = phi0[c];
    double rho = 0.0, kap = 0.0, Sv = 0.0, Gv = 0.0;
    double Ci[MAXSP];
    for (int i = 0; i < MAXSP; ++i) Ci[i] = 0.0;
    if (solvent[c]) {
      double la[MAXSP], u = 0.0;
      if (!fermi_root(sp, ph, u, la)) {
        atomicExch(err, 5);
      } else {
        Sv = u - sp.lgB;
        Gv = exp(u);
        for (int i = 0; i < sp.ns; ++i) {
          Ci[i] = (sp.lvc[i] > -INFINITY) ? exp(sp.lcB[i] - sp.z[i] * ph + sp.p[i] * Sv) : 0.0;
          rho += sp.z[i] * Ci[i];
          kap += sp.lam * sp.z[i] * sp.z[i] * Ci[i];
        }
      }
    }
    if (b1) b1[c] = (solvent[c] && k > 0 && k < nz - 1) ? -sp.lam * rho : 0.0;
    if (sig) sig[c] = kap;
    if (c2) c2[c] = fma(kap, ph, ffix[c]);
    if (C) for (int i = 0; i < sp.ns; ++i) C[i * N + c] = Ci[i];
    if (S) S[c] = Sv;
    if (G) G[c] = Gv;
  }
}

__global__ void k_pf2_rhs(const double* __restrict__ psi, const uint8_t* __restrict__ solvent,
                          const double* __restrict__ c2, double eps_s, double lo, double hi, int nx, int ny, int nz,
                          double* b2) {
  const long N = (long)nx * ny * nz, sxy = (long)nx * ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const long k = c / sxy;
    double v;
    if (k == 0) v = lo;
    else if (k == nz - 1) v = hi;
    else v = (solvent[c] ? -eps_s * psi[c] : 0.0) + c2[c];
    b2[c] = v;
  }
}

__global__ void k_relax(double* __restrict__ phi0, const double* __restrict__ phi, double omega, long n,
                        double* part, unsigned int* ticket, double* delta) {
  double m = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double o = phi0[c];
    const double nw = omega * o + (1.0 - omega) * phi[c];
    m = fmax(m, fabs(nw - o));
    phi0[c] = nw;
  }
  double vals[1] = {m};
  block_partials<1>(vals, 1u, part);
  if (arrive_last(ticket)) {
    double tot[1];
    total_partials<1>(part, 1u, tot);
    if (threadIdx.x == 0) {
      *delta = tot[0];
      *ticket = 0;
    }
  }
}

__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ d, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    x[c] += (double)d[c];
}

// b.b over the two Dirichlet planes (which the stencil kernels do not visit) -> st->bnorm2
__global__ void k_plane_bb(const double* __restrict__ b, int nx, int ny, int nz, BicgState* st) {
  const long plane = (long)nx * ny, N = plane * nz;
  double a = 0.0;
  for (long c = threadIdx.x; c < plane; c += blockDim.x) {
    a = fma(b[c], b[c], a);
    a = fma(b[N - plane + c], b[N - plane + c], a);
  }
  __shared__ double red[NTHREADS];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = NTHREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->bnorm2 = red[0];
}

__global__ void k_scale(const double* __restrict__ a, double s, double* __restrict__ out, long n) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x)
    out[c] = a[c] * s;
}

__global__ void k_set_dirichlet(double* x, double lo, double hi, int nx, int ny, int nz) {
  const long plane = (long)nx * ny, N = plane * nz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < plane; c += (long)gridDim.x * blockDim.x) {
    x[c] = lo;
    x[N - plane + c] = hi;
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

static int ew_blocks(long n) {
  long b = (n + 255) / 256;
  const long cap = (long)nsm() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_faces(const double* eps, int nx, int ny, int nz, double h, double* wE, double* wN, double* wU,
                         double* dsum, cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_faces<<<ew_blocks(N), 256, 0, s>>>(eps, nx, ny, nz, 1.0 / (h * h), wE, wN, wU, dsum);
  return cudaGetLastError();
}

cudaError_t launch_spread(const double* charges, int nq, double ox, double oy, double oz, double h, double lam,
                          int nx, int ny, int nz, double* f, int* err, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  k_spread<<<1, 32, 0, s>>>(charges, nq, ox, oy, oz, h, lam, nx, ny, nz, f, err);
  return cudaGetLastError();
}

cudaError_t launch_eps_diag(const double* dsum, const double* sig, const uint8_t* smask, int nx, int ny, int nz,
                            double* diag, double* dinv, float* dinv32, cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_eps_diag<<<ew_blocks(N), 256, 0, s>>>(dsum, sig, smask, nx, ny, nz, diag, dinv, dinv32);
  return cudaGetLastError();
}

cudaError_t launch_pf1_dinv(const uint8_t* solvent, int nx, int ny, int nz, double dinvc, double* dinv, float* dinv32,
                            cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_pf1_dinv<<<ew_blocks(N), 256, 0, s>>>(solvent, nx, ny, nz, dinvc, dinv, dinv32);
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

template <typename T, bool UNI>
cudaError_t launch_init(const OpView<T>& op, const T* x, bool x_zero, const T* b, T* r, T* rt, T* p, T* v, T* t,
                        double* part, BicgState* st, const Launch& L) {
  k_init<T, UNI><<<L.blocks, NTHREADS, 0, L.stream>>>(op, x, x_zero ? 1 : 0, b, r, rt, p, v, t, part, st, L.ntiles);
  return cudaGetLastError();
}

template <typename T, bool UNI>
cudaError_t launch_phase_b(const OpView<T>& op, const T* r, const T* v, const T* rt, T* t, double* part,
                           BicgState* st, const Launch& L) {
  k_phase_b<T, UNI><<<L.blocks, NTHREADS, 0, L.stream>>>(op, r, v, rt, t, part, st, L.ntiles);
  return cudaGetLastError();
}

template <typename T, bool UNI>
cudaError_t launch_phase_ca(const OpView<T>& op, const T* r, const T* v, const T* p, const T* t, const T* rt, T* x,
                            T* r_out, T* p_out, T* v_out, double* part, BicgState* st, int prime, const Launch& L) {
  k_phase_ca<T, UNI><<<L.blocks, NTHREADS, 0, L.stream>>>(op, r, v, p, t, rt, x, r_out, p_out, v_out, part, st, prime,
                                                          L.ntiles);
  return cudaGetLastError();
}

template <bool UNI>
cudaError_t launch_refine(const OpView<double>& op, double* x, const float* d, const double* b, float* r32,
                          double* part, BicgState* st, const Launch& L) {
  if (d) {
    // x += d is an elementwise pass before the stencil: updating x inside the stencil kernel would race
    // with neighbouring tiles that read x as their halo
    const long N = (long)op.nx * op.ny * op.nz;
    k_add_f32<<<ew_blocks(N), 256, 0, L.stream>>>(x, d, N);
  }
  k_residual<UNI><<<L.blocks, NTHREADS, 0, L.stream>>>(op, x, b, r32, part, st, L.ntiles);
  return cudaGetLastError();
}

cudaError_t launch_fermi(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesParams& sp,
                         int nx, int ny, int nz, double* b1, double* sig, double* c2, double* C, double* S, double* G,
                         int* err, cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_fermi<<<ew_blocks(N), 256, 0, s>>>(phi0, solvent, ffix, sp, nx, ny, nz, b1, sig, c2, C, S, G, err);
  return cudaGetLastError();
}

cudaError_t launch_pf2_rhs(const double* psi, const uint8_t* solvent, const double* c2, double eps_s, double lo,
                           double hi, int nx, int ny, int nz, double* b2, cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_pf2_rhs<<<ew_blocks(N), 256, 0, s>>>(psi, solvent, c2, eps_s, lo, hi, nx, ny, nz, b2);
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

cudaError_t launch_set_dirichlet(double* x, double lo, double hi, int nx, int ny, int nz, cudaStream_t s) {
  k_set_dirichlet<<<ew_blocks((long)nx * ny), 256, 0, s>>>(x, lo, hi, nx, ny, nz);
  return cudaGetLastError();
}

// explicit instantiations
#define PF_INST(T, U)                                                                                              \
  template cudaError_t launch_init<T, U>(const OpView<T>&, const T*, bool, const T*, T*, T*, T*, T*, T*, double*, \
                                         BicgState*, const Launch&);                                               \
  template cudaError_t launch_phase_b<T, U>(const OpView<T>&, const T*, const T*, const T*, T*, double*,          \
                                            BicgState*, const Launch&);                                            \
  template cudaError_t launch_phase_ca<T, U>(const OpView<T>&, const T*, const T*, const T*, const T*, const T*,  \
                                             T*, T*, T*, T*, double*, BicgState*, int, const Launch&);
PF_INST(double, false)
PF_INST(double, true)
PF_INST(float, false)
PF_INST(float, true)
template cudaError_t launch_refine<false>(const OpView<double>&, double*, const float*, const double*, float*,
                                          double*, BicgState*, const Launch&);
template cudaError_t launch_refine<true>(const OpView<double>&, double*, const float*, const double*, float*,
                                         double*, BicgState*, const Launch&);

__global__ void k_set_state(BicgState* st, double tol, int norm, int max_iter) {
  BicgState s = {};
  s.tol = tol;
  s.norm = norm;
  s.max_iter = max_iter;
  *st = s;
}

cudaError_t launch_set_state(BicgState* st, double tol, int norm, int max_iter, cudaStream_t s) {
  k_set_state<<<1, 1, 0, s>>>(st, tol, norm, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_plane_bb(const double* b, int nx, int ny, int nz, BicgState* st, cudaStream_t s) {
  k_plane_bb<<<1, NTHREADS, 0, s>>>(b, nx, ny, nz, st);
  return cudaGetLastError();
}

// Persistent grid size of the stencil kernels: all SMs, as many blocks per SM as every stencil kernel
// can keep resident, never more blocks than tiles.
Launch make_launch(int nx, int ny, int nz, cudaStream_t s) {
  static int per_sm = 0;
  if (!per_sm) {
    int occ = 64, o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_phase_ca<double, false>, NTHREADS, 0); occ = o < occ ? o : occ;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_phase_b<double, false>, NTHREADS, 0); occ = o < occ ? o : occ;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_phase_ca<float, false>, NTHREADS, 0); occ = o < occ ? o : occ;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_phase_b<float, false>, NTHREADS, 0); occ = o < occ ? o : occ;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_init<double, false>, NTHREADS, 0); occ = o < occ ? o : occ;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_residual<false>, NTHREADS, 0); occ = o < occ ? o : occ;
    per_sm = occ > 0 ? occ : 1;
  }
  Launch L;
  L.ntiles = tiles_for(nx, ny, nz);
  L.blocks = nsm() * per_sm;
  if (L.blocks > L.ntiles) L.blocks = L.ntiles;
  L.stream = s;
  return L;
}

int max_partial_blocks() { return nsm() * 16 > 2048 ? nsm() * 16 : 2048; }

}  // namespace pf
