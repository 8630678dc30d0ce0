// pf_kernels.cu -- sm_103a kernels of the Poisson-Fermi hot path.
//
// Stencil kernels (BiCGSTAB phases and the FP64 residual) walk 2D tiles of TX x TY nodes (one warp
// per x row) up through a chunk of ZC interior z-planes.  Every input plane of a tile arrives by
// TMA (cp.async.bulk.tensor.3d) into a ring of D shared-memory stages, each guarded by an mbarrier
// that the copies complete; one thread keeps D planes in flight ahead of the consumers, and the
// stream of planes continues across the tiles a block owns, so the copy engine hides DRAM latency
// without registers.  Arrays read at neighbours arrive as halo boxes (x0-4 .. x0+TX+3, y0-1 ..
// y0+TY: the x start stays 16-byte aligned), the others as centre boxes.  Each plane's stencil input
// (the BiCGSTAB direction p or s after the axpy and the Jacobi scaling) is computed once per node
// into a ring of three shared planes; the planes below and above come from registers.  The axpy
// updates of p, s, x and r (Table 3), the Jacobi scaling and the inner products that give rho, alpha
// and omega are fused into the two stencil kernels of an iteration.  Inner products are reduced by warp
// shuffles, a block tree and the last-arriving block over the per-block partials in fixed order.
#include <math.h>
#include <stdio.h>

#include "pf_internal.cuh"

namespace pf {

// ------------------------------------------------------------------ PTX helpers (TMA + mbarrier)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `limit` clock cycles (the caller then reports PF_E_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

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
// thread's partial sum carries about twice the FP32 precision before the FP64 block reduction.
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

// Inner-product partials of a thread: the products of one tile column (at most ZC + 1 terms) are
// summed in the working precision, then added to an FP64 total once per tile, so the global inner
// products are FP64 sums of short working-precision partial sums.
template <typename T, int NV>
struct Partials {
  T t[NV];
  double d[NV];
  __device__ __forceinline__ Partials() {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      t[j] = T(0);
      d[j] = 0.0;
    }
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      d[j] += (double)t[j];
      t[j] = T(0);
    }
  }
};

// Block reduction of NV values (bit j of maxmask: value j is a maximum, else a sum) into
// part[blockIdx.x * NPART + j]; scratch holds at least NTHREADS / 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], unsigned maxmask, double* part, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double a = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_down_sync(0xffffffffu, a, o);
      a = ((maxmask >> j) & 1u) ? fmax(a, b) : a + b;
    }
    if (lane == 0) scratch[warp * NV + j] = a;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double a = scratch[j];
    for (int w = 1; w < NTHREADS / 32; ++w)
      a = ((maxmask >> j) & 1u) ? fmax(a, scratch[w * NV + j]) : a + scratch[w * NV + j];
    part[blockIdx.x * NPART + j] = a;
  }
}

// True in the block that arrives last; that block then sees every block's partials.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: totals over all blocks' partials in fixed order; scratch holds NTHREADS * NV doubles.
template <int NV>
__device__ __forceinline__ void total_partials(const double* part, unsigned maxmask, double (&tot)[NV],
                                               double* scratch) {
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
  for (int j = 0; j < NV; ++j) scratch[threadIdx.x * NV + j] = a[j];
  __syncthreads();
  for (int s = NTHREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const double u = scratch[threadIdx.x * NV + j], w = scratch[(threadIdx.x + s) * NV + j];
        scratch[threadIdx.x * NV + j] = ((maxmask >> j) & 1u) ? fmax(u, w) : u + w;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = scratch[j];
}

// ------------------------------------------------------------------ tile geometry
int tiles_for(int nx, int ny, int nz) {
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, nzc = (nz - 2 + ZC - 1) / ZC;
  return ntx * nty * nzc;
}

struct Tile {
  int x0, y0, kb, ke;
};

__device__ __forceinline__ Tile tile_of(int t, int nx, int nz) {
  const int nzc = (nz - 2 + ZC - 1) / ZC, ntx = (nx + TX - 1) / TX;
  const int zc = t % nzc, xy = t / nzc;
  Tile r;
  r.x0 = (xy % ntx) * TX;
  r.y0 = (xy / ntx) * TY;
  r.kb = 1 + zc * ZC;
  r.ke = min(r.kb + ZC, nz - 1);
  return r;
}

// Position g in [-1, n] -> the node whose value it holds: itself, the mirror image for the two ghost
// positions of the zero-flux sides (Eq. 4), or -1 when no output of the tile uses it.
__device__ __forceinline__ int mirror(int g, int n) {
  if (g < 0) return 1;
  if (g < n) return g;
  if (g == n) return n - 2;
  return -1;
}

constexpr int PW = TX + 2;             // shared stencil-plane row pitch
constexpr int PLANE = (TY + 2) * PW;   // shared stencil-plane size
constexpr int NHALO = 2 * (TX + 2) + 2 * TY;

__device__ __forceinline__ int cs(int lx, int ly) { return (ly + 1) * PW + (lx + 1); }

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

// Per-thread geometry of a tile: halo-box offsets of the thread's centre and of its halo slot (with
// the mirror applied), the shared-plane index of the halo slot, and whether the centre is a node.
struct TileGeo {
  int cbo;    // halo-box offset of the centre position, -1 if unused
  int hbo;    // halo-box offset of the halo slot's position, -1 if unused
  int hs;     // shared-plane index of the halo slot, -1 if the thread has none
  int gi, gj;
  bool valid;
};

__device__ __forceinline__ int box_off(int gi, int gj, const Tile& tl, int nx, int ny) {
  const int mi = mirror(gi, nx), mj = mirror(gj, ny);
  if (mi < 0 || mj < 0) return -1;
  return (mj - tl.y0 + 1) * HBX + (mi - tl.x0 + 4);
}

__device__ __forceinline__ TileGeo tile_geo(const Tile& tl, int nx, int ny) {
  TileGeo g;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  g.gi = tl.x0 + lx;
  g.gj = tl.y0 + ly;
  g.valid = g.gi < nx && g.gj < ny;
  g.cbo = box_off(g.gi, g.gj, tl, nx, ny);
  g.hbo = -1;
  g.hs = -1;
  // the halo slots go to the last NHALO threads, away from the producer thread in warp 0
  const int hslot = (int)threadIdx.x - (NTHREADS - NHALO);
  if (hslot >= 0) {
    int hx, hy;
    halo_pos(hslot, hx, hy);
    g.hs = cs(hx, hy);
    g.hbo = box_off(tl.x0 + hx, tl.y0 + hy, tl, nx, ny);
  }
  return g;
}

template <typename T>
__host__ __device__ constexpr int halo_slot_bytes() {
  return (HBX * HBY * (int)sizeof(T) + 127) / 128 * 128;
}
template <typename T>
__host__ __device__ constexpr int centre_slot_bytes() {
  return TX * TY * (int)sizeof(T);
}

template <class Op>
__host__ __device__ constexpr int stage_bytes() {
  return Op::NH * halo_slot_bytes<typename Op::T>() + Op::NC * centre_slot_bytes<typename Op::T>();
}

template <class Op>
__host__ __device__ constexpr int smem_bytes() {
  // stages | three stencil planes | D mbarriers | 128 bytes of alignment slack
  return Op::D * stage_bytes<Op>() + 3 * PLANE * (int)sizeof(typename Op::T) + Op::D * 8 + 128;
}

// The reduction scratch at the end of a kernel reuses the stage ring (all copies consumed by then).
template <class Op>
constexpr bool scratch_fits() {
  return Op::D * stage_bytes<Op>() >= NTHREADS * 8 * (int)sizeof(double);
}

// ------------------------------------------------------------------ the pipelined stencil kernel
// Op supplies: T, NH, NC, D, CHECK_DONE, Args, Sc, Ctr, Accs and scalars(), q_of(), centre(),
// up_face(), output(), finish().
template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB) k_stencil(const __grid_constant__ Maps<Op::NH, Op::NC> maps,
                                                      typename Op::Args a, Geom g, int ntiles,
                                                      unsigned long long wait_limit) {
  using T = typename Op::T;
  constexpr int D = Op::D, NH = Op::NH, NC = Op::NC;
  constexpr int HB = halo_slot_bytes<T>(), CB = centre_slot_bytes<T>(), STAGE = stage_bytes<Op>();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  T* qring = reinterpret_cast<T*>(smem + D * STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + D * STAGE + 3 * PLANE * sizeof(T));

  if (Op::CHECK_DONE && *(volatile int*)&a.st->done) return;
  const typename Op::Sc sc = Op::scalars(a);
  if (threadIdx.x == 0) {
    for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producer (thread 0): the next (tile, plane) of this block's stream of planes
  static_assert((D & (D - 1)) == 0, "the stage ring has a power-of-two size");
  int pt = blockIdx.x, pj = 0;
  unsigned pseq = 0;
  Tile ptl = tile_of(pt, g.nx, g.nz);
  auto issue = [&]() {
    const int stage = pseq & (D - 1);
    unsigned char* sb = smem + stage * STAGE;
    uint64_t* bar = &bars[stage];
    mbar_expect_tx(bar, NH * HBX * HBY * sizeof(T) + NC * TX * TY * sizeof(T));
    const int k = ptl.kb - 1 + pj;
#pragma unroll
    for (int h = 0; h < NH; ++h) tma_load_3d(sb + h * HB, &maps.h[h], ptl.x0 - 4, ptl.y0 - 1, k, bar);
#pragma unroll
    for (int c = 0; c < NC; ++c) tma_load_3d(sb + NH * HB + c * CB, &maps.c[c], ptl.x0, ptl.y0, k, bar);
    ++pseq;
    if (++pj == ptl.ke - ptl.kb + 2) {
      pj = 0;
      pt += gridDim.x;
      if (pt < ntiles) ptl = tile_of(pt, g.nx, g.nz);
    }
  };
  if (threadIdx.x == 0)
    for (int d = 0; d < D && pt < ntiles; ++d) issue();

  typename Op::Accs acc;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  unsigned seq = 0;
  bool failed = false;
  for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    const Tile tl = tile_of(t, g.nx, g.nz);
    const TileGeo geo = tile_geo(tl, g.nx, g.ny);
    const int planes = tl.ke - tl.kb + 2;
    typename Op::Ctr cprev{}, cnow{};
    T q_dn = T(0), q_prev = T(0), wD = T(0);
    T* Qnow = qring;                 // plane j
    T* Qprev = qring + 2 * PLANE;    // plane j-1
    T* Qold = qring + PLANE;         // plane j-2 (free for plane j+1)
    long cidx = geo.gi + (long)g.px * geo.gj + g.plane * (tl.kb - 1);
    for (int j = 0; j < planes; ++j, ++seq) {
      const int stage = seq & (D - 1);
      const bool ok = mbar_wait(&bars[stage], (seq / D) & 1u, wait_limit);
      T qc = T(0);
      if (ok) {
        const unsigned char* sb = smem + stage * STAGE;
        const T* H[NH];
        const T* C[NC];
#pragma unroll
        for (int h = 0; h < NH; ++h) H[h] = reinterpret_cast<const T*>(sb + h * HB);
#pragma unroll
        for (int c = 0; c < NC; ++c) C[c] = reinterpret_cast<const T*>(sb + NH * HB + c * CB);
        if (geo.cbo >= 0) qc = Op::q_of(sc, H, geo.cbo, &cnow);
        if (geo.valid) Op::centre(a, H, C, geo.cbo, ly * TX + lx, geo.gi > 0, geo.gj > 0, cnow);
        Qnow[cs(lx, ly)] = qc;
        if (geo.hs >= 0) Qnow[geo.hs] = geo.hbo >= 0 ? Op::q_of(sc, H, geo.hbo, nullptr) : T(0);
      }
      // one barrier per plane; the vote makes a timed-out wait a decision of the whole block
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (threadIdx.x == 0 && pt < ntiles) {
        fence_proxy_async();
        issue();
      }
      if (j >= 2 && geo.valid) Op::output(sc, a, Qprev, lx, ly, cidx, cprev, q_dn, qc, wD, acc);
      if (j >= 1) {
        q_dn = q_prev;
        wD = Op::up_face(a, cprev);
        cidx += g.plane;
      }
      q_prev = qc;
      cprev = cnow;
      // rotate the three stencil planes
      T* const freed = Qold;
      Qold = Qprev;
      Qprev = Qnow;
      Qnow = freed;
    }
    acc.flush();
    if (!failed) __syncthreads();
  }
  if (failed) {
    // give up: let this block's copies in flight land (bounded), report the timeout, skip the reduction
    if (threadIdx.x == 0) {
      for (unsigned s = seq; s < pseq; ++s) mbar_wait(&bars[s & (D - 1)], (s / D) & 1u, wait_limit);
      a.st->status = 7;  // PF_E_TIMEOUT
      atomicExch(&a.st->done, 1);
    }
    return;
  }
  __syncthreads();
  Op::finish(a, acc, reinterpret_cast<double*>(smem));
}

// ------------------------------------------------------------------ phase B: s = r - alpha v, t = A M^-1 s
template <typename T_, bool UNI>
struct OpB {
  using T = T_;
  static constexpr int NH = SlotsB<UNI>::NH, NC = SlotsB<UNI>::NC, D = sizeof(T_) == 4 ? 4 : 2;
  static constexpr int MINB = sizeof(T_) == 4 ? 4 : 2;
  static constexpr bool CHECK_DONE = true;
  enum { R = 0, V = 1, DI = 2, WE = 3, WN = 4 };
  enum { RT = 0, WU = 1 };
  struct Args {
    double* part;
    BicgState* st;
    T* t;
    T wc;
  };
  struct Sc {
    T al;
  };
  struct Ctr {
    T s, di, rt, wU, wEc, wEw, wNc, wNs;
  };
  struct Accs {
    Partials<T, 5> p;  // r~.s, r~.t, t.s, t.t, s.s
    T smax = T(0);
    __device__ void flush() { p.flush(); }
  };
  __device__ static Sc scalars(const Args& a) { return Sc{(T)a.st->alpha}; }
  __device__ static T q_of(const Sc& sc, const T* const* H, int o, Ctr* c) {
    const T s = fma(-sc.al, H[V][o], H[R][o]);
    const T di = H[DI][o];
    if (c) {
      c->s = s;
      c->di = di;
    }
    return di * s;
  }
  __device__ static void centre(const Args& a, const T* const* H, const T* const* C, int o, int co, bool west,
                                bool south, Ctr& c) {
    c.rt = C[RT][co];
    if (UNI) {
      c.wU = c.wEc = c.wEw = c.wNc = c.wNs = a.wc;
    } else {
      c.wU = C[WU][co];
      c.wEc = H[WE][o];
      c.wEw = west ? H[WE][o - 1] : c.wEc;
      c.wNc = H[WN][o];
      c.wNs = south ? H[WN][o - HBX] : c.wNc;
    }
  }
  __device__ static T up_face(const Args& a, const Ctr& c) { return UNI ? a.wc : c.wU; }
  __device__ static void output(const Sc&, const Args& a, const T* Q, int lx, int ly, long cidx, const Ctr& c, T q_dn,
                                T q_up, T wD, Accs& acc) {
    T tc;
    if (c.di == T(0)) {
      tc = c.s;
    } else {
      const T qE = Q[cs(lx + 1, ly)], qW = Q[cs(lx - 1, ly)], qN = Q[cs(lx, ly + 1)], qS = Q[cs(lx, ly - 1)];
      T nb;
      if (UNI) {
        nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        nb = c.wEc * qE;
        nb = fma(c.wEw, qW, nb);
        nb = fma(c.wNc, qN, nb);
        nb = fma(c.wNs, qS, nb);
        nb = fma(c.wU, q_up, nb);
        nb = fma(wD, q_dn, nb);
      }
      tc = c.s - nb;
    }
    a.t[cidx] = tc;
    acc.p.t[0] = fma(c.rt, c.s, acc.p.t[0]);
    acc.p.t[1] = fma(c.rt, tc, acc.p.t[1]);
    acc.p.t[2] = fma(tc, c.s, acc.p.t[2]);
    acc.p.t[3] = fma(tc, tc, acc.p.t[3]);
    acc.p.t[4] = fma(c.s, c.s, acc.p.t[4]);
    acc.smax = fmax(acc.smax, tabs(c.s));
  }
  __device__ static void finish(const Args& a, const Accs& acc, double* scratch) {
    double vals[6] = {acc.p.d[0], acc.p.d[1], acc.p.d[2], acc.p.d[3], acc.p.d[4], (double)acc.smax};
    block_partials<6>(vals, 32u, a.part, scratch);
    if (!arrive_last(&a.st->ticket)) return;
    double tot[6];
    total_partials<6>(a.part, 32u, tot, scratch);
    if (threadIdx.x != 0) return;
    BicgState* st = a.st;
    const double rs = tot[0], rtt = tot[1], ts = tot[2], tt = tot[3], ss = tot[4], smx = tot[5];
    st->snorm2 = ss;
    st->sinf = smx;
    const bool sconv = st->norm == 0 ? (ss <= st->tol2) : (smx < st->tol);
    if (sconv) {  // early exit of the Templates algorithm: x += alpha M^-1 p, r = s
      st->sexit = 1;
      st->omega = 0.0;
      st->beta = 0.0;
    } else if (tt == 0.0 || !isfinite(tt) || !isfinite(ts) || !isfinite(ss)) {
      st->status = 4;  // PF_E_BREAKDOWN, before x is touched
      st->done = 1;
    } else {
      const double om = ts / tt;  // omega = t.s / t.t
      st->omega = om;
      // r~.r_new with r_new = s - omega t (the next rho): the next p is
      // formed in the same kernel as r_new, so its beta is taken from the exact identity
      const double rho_new = rs - om * rtt;
      const double be = (om != 0.0) ? (rho_new / st->rho) * (st->alpha / om) : 0.0;  // beta
      st->beta = isfinite(be) ? be : 0.0;
    }
    st->ticket = 0;
  }
};

// ------------------------------------------------------------------ phase C+A
// s = r - alpha v, x += alpha M^-1 p + omega M^-1 s, r' = s - omega t, and for the next iteration
// p' = r' + beta (p - omega v) and v' = A M^-1 p'.
template <typename T_, bool UNI>
struct OpCA {
  using T = T_;
  static constexpr int NH = SlotsCA<UNI>::NH, NC = SlotsCA<UNI>::NC, D = 2;
  static constexpr int MINB = sizeof(T_) == 4 ? 4 : 2;
  static constexpr bool CHECK_DONE = true;
  enum { R = 0, V = 1, TT = 2, P = 3, DI = 4, WE = 5, WN = 6 };
  enum { X = 0, RT = 1, WU = 2 };
  struct Args {
    double* part;
    BicgState* st;
    T* x;
    T* r_out;
    T* p_out;
    T* v_out;
    T wc;
    int prime;
  };
  struct Sc {
    T al, om, be;
  };
  struct Ctr {
    T s, rn, pn, pold, di, x, rt, wU, wEc, wEw, wNc, wNs;
  };
  struct Accs {
    Partials<T, 3> p;  // r~.v', r~.r', r'.r'
    T rmax = T(0);
    __device__ void flush() { p.flush(); }
  };
  __device__ static Sc scalars(const Args& a) { return Sc{(T)a.st->alpha, (T)a.st->omega, (T)a.st->beta}; }
  __device__ static T q_of(const Sc& sc, const T* const* H, int o, Ctr* c) {
    const T vv = H[V][o], pp = H[P][o];
    const T s = fma(-sc.al, vv, H[R][o]);
    const T rn = fma(-sc.om, H[TT][o], s);
    const T pn = fma(sc.be, fma(-sc.om, vv, pp), rn);
    const T di = H[DI][o];
    if (c) {
      c->s = s;
      c->rn = rn;
      c->pn = pn;
      c->pold = pp;
      c->di = di;
    }
    return di * pn;
  }
  __device__ static void centre(const Args& a, const T* const* H, const T* const* C, int o, int co, bool west,
                                bool south, Ctr& c) {
    c.x = C[X][co];
    c.rt = C[RT][co];
    if (UNI) {
      c.wU = c.wEc = c.wEw = c.wNc = c.wNs = a.wc;
    } else {
      c.wU = C[WU][co];
      c.wEc = H[WE][o];
      c.wEw = west ? H[WE][o - 1] : c.wEc;
      c.wNc = H[WN][o];
      c.wNs = south ? H[WN][o - HBX] : c.wNc;
    }
  }
  __device__ static T up_face(const Args& a, const Ctr& c) { return UNI ? a.wc : c.wU; }
  __device__ static void output(const Sc& sc, const Args& a, const T* Q, int lx, int ly, long cidx, const Ctr& c,
                                T q_dn, T q_up, T wD, Accs& acc) {
    T vn;
    if (c.di == T(0)) {
      vn = c.pn;
    } else {
      const T qE = Q[cs(lx + 1, ly)], qW = Q[cs(lx - 1, ly)], qN = Q[cs(lx, ly + 1)], qS = Q[cs(lx, ly - 1)];
      T nb;
      if (UNI) {
        nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        nb = c.wEc * qE;
        nb = fma(c.wEw, qW, nb);
        nb = fma(c.wNc, qN, nb);
        nb = fma(c.wNs, qS, nb);
        nb = fma(c.wU, q_up, nb);
        nb = fma(wD, q_dn, nb);
      }
      vn = c.pn - nb;
      if (!a.prime) {
        T xc = fma(sc.al, c.di * c.pold, c.x);
        xc = fma(sc.om, c.di * c.s, xc);
        a.x[cidx] = xc;
      }
    }
    a.r_out[cidx] = c.rn;
    a.p_out[cidx] = c.pn;
    a.v_out[cidx] = vn;
    acc.p.t[0] = fma(c.rt, vn, acc.p.t[0]);
    acc.p.t[1] = fma(c.rt, c.rn, acc.p.t[1]);
    acc.p.t[2] = fma(c.rn, c.rn, acc.p.t[2]);
    acc.rmax = fmax(acc.rmax, tabs(c.rn));
  }
  __device__ static void finish(const Args& a, const Accs& acc, double* scratch) {
    double vals[4] = {acc.p.d[0], acc.p.d[1], acc.p.d[2], (double)acc.rmax};
    block_partials<4>(vals, 8u, a.part, scratch);
    if (!arrive_last(&a.st->ticket)) return;
    double tot[4];
    total_partials<4>(a.part, 8u, tot, scratch);
    if (threadIdx.x != 0) return;
    BicgState* st = a.st;
    const double rv = tot[0], rr = tot[1], r2 = tot[2], rmx = tot[3];
    st->ticket = 0;
    if (!a.prime) {
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
    st->rho = rr;         // rho of the next iteration
    st->alpha = rr / rv;  // alpha of the next iteration
  }
};

// Squared 2-norm stop of a state whose residual has squared norm rr and right-hand side bb: the first
// residual of a solve fixes r0norm2; the threshold is the larger of the b-relative and r0-relative ones.
__device__ __forceinline__ void set_tol2(BicgState* st, double rr, double bb) {
  if (!(st->r0norm2 >= 0.0)) st->r0norm2 = rr;
  st->tol2 = fmax(st->tol * st->tol * bb, st->tol_r0 * st->tol_r0 * st->r0norm2);
}

// ------------------------------------------------------------------ FP64 residual b - A x
template <bool UNI>
struct OpRes {
  using T = double;
  static constexpr int NH = SlotsRes<UNI>::NH, NC = SlotsRes<UNI>::NC, D = 2;
  static constexpr int MINB = 2;
  static constexpr bool CHECK_DONE = false;
  enum { X = 0, DI = 1, WE = 2, WN = 3 };
  enum { B = 0, DG = 1, WU = 2 };
  struct Args {
    double* part;
    BicgState* st;
    double wc, diagc;
    int init;
    double *r, *rt, *p, *v, *t;
    float* r32;
  };
  struct Sc {
    int unused;
  };
  struct Ctr {
    double xc, di, b, diag, wU, wEc, wEw, wNc, wNs;
  };
  struct Accs {
    double rr = 0.0, bb = 0.0, rmax = 0.0;
    __device__ void flush() {}
  };
  __device__ static Sc scalars(const Args&) { return Sc{0}; }
  __device__ static double q_of(const Sc&, const double* const* H, int o, Ctr* c) {
    const double xv = H[X][o];
    if (c) {
      c->xc = xv;
      c->di = H[DI][o];
    }
    return xv;
  }
  __device__ static void centre(const Args& a, const double* const* H, const double* const* C, int o, int co,
                                bool west, bool south, Ctr& c) {
    c.b = C[B][co];
    if (UNI) {
      c.diag = a.diagc;
      c.wU = c.wEc = c.wEw = c.wNc = c.wNs = a.wc;
    } else {
      c.diag = C[DG][co];
      c.wU = C[WU][co];
      c.wEc = H[WE][o];
      c.wEw = west ? H[WE][o - 1] : c.wEc;
      c.wNc = H[WN][o];
      c.wNs = south ? H[WN][o - HBX] : c.wNc;
    }
  }
  __device__ static double up_face(const Args& a, const Ctr& c) { return UNI ? a.wc : c.wU; }
  __device__ static void output(const Sc&, const Args& a, const double* Q, int lx, int ly, long cidx, const Ctr& c,
                                double q_dn, double q_up, double wD, Accs& acc) {
    double rc;
    if (c.di == 0.0) {
      rc = c.b - c.xc;
    } else {
      const double qE = Q[cs(lx + 1, ly)], qW = Q[cs(lx - 1, ly)], qN = Q[cs(lx, ly + 1)], qS = Q[cs(lx, ly - 1)];
      double nb;
      if (UNI) {
        nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        nb = c.wEc * qE;
        nb = fma(c.wEw, qW, nb);
        nb = fma(c.wNc, qN, nb);
        nb = fma(c.wNs, qS, nb);
        nb = fma(c.wU, q_up, nb);
        nb = fma(wD, q_dn, nb);
      }
      rc = c.b - (c.diag * c.xc - nb);
    }
    if (a.init) {
      a.r[cidx] = rc;
      a.rt[cidx] = rc;
      a.p[cidx] = 0.0;
      a.v[cidx] = 0.0;
      a.t[cidx] = 0.0;
    } else {
      a.r32[cidx] = (float)rc;
    }
    acc.rr = fma(rc, rc, acc.rr);
    acc.bb = fma(c.b, c.b, acc.bb);
    acc.rmax = fmax(acc.rmax, fabs(rc));
  }
  __device__ static void finish(const Args& a, const Accs& acc, double* scratch) {
    double vals[3] = {acc.rr, acc.bb, acc.rmax};
    block_partials<3>(vals, 4u, a.part, scratch);
    if (!arrive_last(&a.st->ticket)) return;
    double tot[3];
    total_partials<3>(a.part, 4u, tot, scratch);
    if (threadIdx.x != 0) return;
    BicgState* st = a.st;
    double bb = tot[1] + st->bnorm2;  // bnorm2 was preset to b.b over the Dirichlet planes
    if (bb == 0.0) bb = 1.0;
    st->bnorm2 = bb;
    st->rnorm2 = tot[0];
    st->rinf = tot[2];
    set_tol2(st, tot[0], bb);
    const bool conv = st->norm == 0 ? (tot[0] <= st->tol2) : (tot[2] < st->tol);
    if (a.init) {
      st->rho = tot[0];  // r~ = r0
      st->alpha = st->omega = st->beta = 0.0;
      st->sexit = 0;
      st->iter = 0;
      st->status = 0;
    }
    st->done = conv ? 1 : 0;
    st->ticket = 0;
  }
};

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
                        double* dsum) {
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

// b.b over the two Dirichlet planes (which the stencil kernels do not visit) -> st->bnorm2
__global__ void k_plane_bb(const double* __restrict__ b, Geom g, BicgState* st) {
  double a = 0.0;
  const long last = g.plane * (g.nz - 1);
  for (long r = 0; r < g.ny; ++r)
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const double u = b[i + g.px * r], w = b[last + i + g.px * r];
      a = fma(u, u, a);
      a = fma(w, w, a);
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

__global__ void k_set_state(BicgState* st, double tol, int norm, int max_iter, double tol_r0, int keep_r0) {
  const double r0 = keep_r0 ? st->r0norm2 : -1.0;
  BicgState s = {};
  s.tol = tol;
  s.norm = norm;
  s.max_iter = max_iter;
  s.tol_r0 = tol_r0;
  s.r0norm2 = r0;
  *st = s;
}


// ------------------------------------------------------------------ Eq. (1) pointwise step
// With la_i = ln(v_i cB_i) - z_i phi - p_i ln Gamma^B, the void fraction Gamma = e^u solves
//   f(u) = e^u + sum_i exp(la_i + p_i u) - 1 = 0,
// f increasing; every term is at most 1 on the bracket [lo, hi] below, so nothing overflows there.
// Newton runs first in FP32 on du = u - u0 (u0: the previous outer iterate's root, or ln Gamma^B), then in
// FP64 until the step is below 1e-8 |u|; as Newton converges quadratically the last FP64 step leaves u
// exact to rounding, and the concentrations come from the last FP64 terms, term_i = v_i C_i, moved to the
// final u by exp(p_i du) = 1 + p_i du + (p_i du)^2/2.
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
    if (fabs(du) <= 1e-8 * fmax(1.0, fabs(u))) {  // converged: take the last Newton step and finish
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

// ulast holds each node's ln Gamma from the previous call (warm != 0) and receives the new one.
__global__ void k_fermi(const double* __restrict__ phi0, const uint8_t* __restrict__ solvent,
                        const double* __restrict__ ffix, SpeciesParams sp, Geom g, double* b1, double* sig, double* c2,
                        double* C, double* S, double* G, double* ulast, int warm, int* err) {
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
      ok = fermi_point(sp, ph, warm ? ulast[c] : sp.lgB, fo);
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

static int row_blocks(const Geom& g) {
  long b = (long)g.ny * g.nz;
  const long cap = (long)nsm() * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

bool encode_map(CUtensorMap* m, const void* base, const Geom& g, int elem_bytes, bool halo) {
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
  const cuuint32_t box[3] = {(cuuint32_t)(halo ? HBX : TX), (cuuint32_t)(halo ? HBY : TY), 1};
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
cudaError_t launch_phase_b(const Maps<SlotsB<UNI>::NH, SlotsB<UNI>::NC>& m, const Geom& g, T wc, T* t, double* part,
                           BicgState* st, const Launch& L) {
  typename OpB<T, UNI>::Args a{part, st, t, wc};
  return launch_stencil<OpB<T, UNI>>(m, a, g, L);
}

template <typename T, bool UNI>
cudaError_t launch_phase_ca(const Maps<SlotsCA<UNI>::NH, SlotsCA<UNI>::NC>& m, const Geom& g, T wc, T* x, T* r_out,
                            T* p_out, T* v_out, double* part, BicgState* st, int prime, const Launch& L) {
  typename OpCA<T, UNI>::Args a{part, st, x, r_out, p_out, v_out, wc, prime};
  return launch_stencil<OpCA<T, UNI>>(m, a, g, L);
}

template <bool UNI>
cudaError_t launch_residual(const Maps<SlotsRes<UNI>::NH, SlotsRes<UNI>::NC>& m, const Geom& g, double wc,
                            double diagc, int init, double* r, double* rt, double* p, double* v, double* t, float* r32,
                            double* part, BicgState* st, const Launch& L) {
  typename OpRes<UNI>::Args a{part, st, wc, diagc, init, r, rt, p, v, t, r32};
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

cudaError_t launch_plane_bb(const double* b, const Geom& g, BicgState* st, cudaStream_t s) {
  k_plane_bb<<<1, NTHREADS, 0, s>>>(b, g, st);
  return cudaGetLastError();
}

cudaError_t launch_faces(const double* eps, const Geom& g, double h, double* wE, double* wN, double* wU, double* dsum,
                         cudaStream_t s) {
  k_faces<<<row_blocks(g), 128, 0, s>>>(eps, g, 1.0 / (h * h), wE, wN, wU, dsum);
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
                         double* ulast, int warm, int* err, cudaStream_t s) {
  k_fermi<<<ew_blocks(g.np), 256, 0, s>>>(phi0, solvent, ffix, sp, g, b1, sig, c2, C, S, G, ulast, warm, err);
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
  template cudaError_t launch_phase_b<T, U>(const Maps<SlotsB<U>::NH, SlotsB<U>::NC>&, const Geom&, T, T*, double*, \
                                            BicgState*, const Launch&);                                            \
  template cudaError_t launch_phase_ca<T, U>(const Maps<SlotsCA<U>::NH, SlotsCA<U>::NC>&, const Geom&, T, T*, T*,   \
                                             T*, T*, double*, BicgState*, int, const Launch&);
PF_INST(double, false)
PF_INST(double, true)
PF_INST(float, false)
PF_INST(float, true)
template cudaError_t launch_residual<false>(const Maps<SlotsRes<false>::NH, SlotsRes<false>::NC>&, const Geom&, double,
                                            double, int, double*, double*, double*, double*, double*, float*, double*,
                                            BicgState*, const Launch&);
template cudaError_t launch_residual<true>(const Maps<SlotsRes<true>::NH, SlotsRes<true>::NC>&, const Geom&, double,
                                           double, int, double*, double*, double*, double*, double*, float*, double*,
                                           BicgState*, const Launch&);
template cudaError_t launch_init_zero<float>(const float*, const Geom&, float*, float*, float*, float*, float*, double*,
                                             BicgState*, cudaStream_t);
template cudaError_t launch_init_zero<double>(const double*, const Geom&, double*, double*, double*, double*, double*,
                                              double*, BicgState*, cudaStream_t);

}  // namespace pf

// ====================================================================================================
// Entry point that allocates nothing: the pointwise Fermi/steric step of Eq. (1) on caller arrays.
//
// Some callers cannot allocate device memory at the moment they need this step: a host application
// that hands the library a fixed device arena, or code that runs where cudaMalloc is not allowed or
// would stall (a memory pool owned by another runtime, a latency-critical loop).  This variant of
// k_fermi keeps its scratch -- each node's ln Gamma and the root-failure flag -- in a file-scope device
// array of fixed size instead of in a pf_grid, so a call needs only the caller's input and output
// arrays.  The paper has no counterpart: it is a property of this library's interface only.
// ====================================================================================================
#include <mutex>

#include "../../include/pf_gb300.h"

void pf_internal_set_error(const char* msg);  // pf_api.cu: the message pf_last_error returns

namespace pf {

// scratch: PF_FERMI_NOALLOC_MAX_NODES doubles of ln Gamma, then the failure flag (one 8-byte word)
static __device__ __align__(256) double g_fermi_scratch[PF_FERMI_NOALLOC_MAX_NODES + 1];

// Same arithmetic as k_fermi: phi arrives in volts (phi_hat = phi * inv_tv), C leaves in mol/L; arrays are
// compact (x fastest, N = n entries per field).
__global__ void k_fermi_noalloc(const double* __restrict__ phi_V, const uint8_t* __restrict__ solvent, long n,
                                SpeciesParams sp, double inv_tv, double inv_molar, double* C, double* S, double* G,
                                double* scratch) {
  double* ulast = scratch;
  unsigned long long* flag = reinterpret_cast<unsigned long long*>(scratch + PF_FERMI_NOALLOC_MAX_NODES);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const double ph = phi_V[c] * inv_tv;
    const bool sol = solvent[c] != 0;
    FermiOut fo;
    bool ok = false;
    if (sol) {
      ok = fermi_point(sp, ph, sp.lgB, fo);
      if (!ok) atomicExch(flag, 1ull);
      else ulast[c] = fo.u;
    }
    for (int s = 0; s < sp.ns; ++s)
      if (C) C[s * n + c] = (sol && ok) ? fo.C[s] * inv_molar : 0.0;
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
                           const pf_species* species, double T_K, double* C_M, double* S, double* Gamma,
                           void* cuda_stream) {
  using namespace pf;
  if (n < 1 || n > PF_FERMI_NOALLOC_MAX_NODES)
    return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: n must be between 1 and PF_FERMI_NOALLOC_MAX_NODES");
  if (!phi_V || !solvent || !species || n_species < 1 || n_species > PF_MAX_SPECIES || !(T_K > 0))
    return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: bad arguments");
  // species constants of Eq. (1), as pf_set_coeffs computes them (Table 1 constants)
  const double kb = 1.38e-23, qe = 1.602e-19, eps0 = 8.85e-12, molar = 6.02214076e23 * 1e-27;
  SpeciesParams sp{};
  double v[PF_MAX_SPECIES], v0 = 0.0, gB = 1.0, q = 0.0, qs = 0.0;
  for (int i = 0; i < n_species; ++i) {
    if (!(species[i].radius_A > 0) || !(species[i].bulk_M >= 0))
      return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: species need radius > 0 and bulk >= 0");
    v[i] = 4.0 * M_PI * species[i].radius_A * species[i].radius_A * species[i].radius_A / 3.0;
    v0 += v[i];
  }
  v0 /= n_species;
  sp.ns = n_species;
  for (int i = 0; i < n_species; ++i) {
    const double cB = species[i].bulk_M * molar;
    sp.z[i] = species[i].z;
    sp.p[i] = v[i] / v0;
    sp.lvc[i] = cB > 0 ? log(v[i] * cB) : -INFINITY;
    sp.lcB[i] = cB > 0 ? log(cB) : -INFINITY;
    sp.inv_v[i] = 1.0 / v[i];
    sp.inv_p[i] = 1.0 / sp.p[i];
    if (cB > 0) sp.lnn += 1.0;
    gB -= v[i] * cB;
    q += species[i].z * cB;
    qs += fabs((double)species[i].z) * cB;
  }
  if (!(gB > 0)) return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: bulk void fraction Gamma^B <= 0");
  if (fabs(q) > 1e-12 * (qs > 0 ? qs : 1.0)) return noalloc_fail(PF_E_INVAL, "pf_fermi_noalloc: bath not neutral");
  sp.lgB = log(gB);
  sp.lnn = log(1.0 + sp.lnn);
  sp.lam = qe * qe / (eps0 * kb * T_K * 1e-10);
  const double tv = kb * T_K / qe;

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
  // the failure flag must start at zero; the ln Gamma part is written before it is read
  if (cudaMemsetAsync(scratch + PF_FERMI_NOALLOC_MAX_NODES, 0, sizeof(double), s) != cudaSuccess)
    return noalloc_fail(PF_E_CUDA, "pf_fermi_noalloc: clearing the flag failed");
  long blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_fermi_noalloc<<<(int)blocks, 256, 0, s>>>(phi_V, solvent, n, sp, 1.0 / tv, 1.0 / molar, C_M, S, Gamma, scratch);
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
