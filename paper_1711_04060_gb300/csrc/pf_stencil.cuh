// pf_stencil.cuh -- the TMA-pipelined 7-point stencil body and the BiCGSTAB / residual operators that
// run on it, shared by the single-grid kernels (pf_kernels.cu) and the batched kernels (pf_batch.cu).
//
// A stencil body walks 2D tiles of TX x TY nodes (one warp per x row) up through a chunk of ZC interior
// z-planes.  Every input plane of a tile arrives by TMA (cp.async.bulk.tensor.3d) into a ring of D
// shared-memory stages, each guarded by an mbarrier that the copies complete; one thread keeps D planes
// in flight ahead of the consumers, and the stream of planes continues across the tiles a block owns, so
// the copy engine hides DRAM latency without registers.  Arrays read at neighbours arrive as halo boxes (x0-4 ..
// x0+TX+3, y0-1 .. y0+TY: the x start stays 16-byte aligned), the others as the same box without its first and
// last row.  On a grid whose x (y) extent is one more than a multiple of TX (TY) the last column (row) can go
// without a tile of its own: the threads whose halo slots hold those nodes in the tile next to them also compute
// them (edge nodes), keeping their per-plane state in shared memory; such a grid loads every array as a halo box.
// Each plane's stencil input (the BiCGSTAB direction p or s after the axpy and the Jacobi scaling) is computed
// once per node into a ring of three shared planes; the planes below and above come from registers.  The
// axpy updates of p, s, x and r (Table 3), the Jacobi scaling and the inner products that give rho, alpha
// and omega are fused into the two stencil kernels of an iteration.  Inner products are reduced by warp
// shuffles, a block tree and the last-arriving block over the per-block partials in fixed order.
#pragma once
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

// Inner-product partials: a thread sums the products of one tile column (at most zc + 1 terms) in the
// working precision; at the end of each tile the warp adds its threads' sums in FP64 (fixed shuffle tree)
// to its FP64 totals in shared memory (wsum[warp * NV + j]), so the global inner products are FP64 sums of
// short working-precision partial sums and no thread holds FP64 accumulators across tiles.
template <typename T, int NV>
struct Partials {
  T t[NV];
  __device__ __forceinline__ Partials() {
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] = T(0);
  }
  // all 32 lanes of the warp take part
  __device__ __forceinline__ void flush(double* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double v = (double)t[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[warp * NV + j] += v;
      t[j] = T(0);
    }
  }
  // the warp's total j (lane 0; 0 on the other lanes), once every tile is flushed
  __device__ __forceinline__ static double total(const double* wsum, int j) {
    return (threadIdx.x & 31) == 0 ? wsum[(threadIdx.x >> 5) * NV + j] : 0.0;
  }
};

// FP32 kernels: GB300's FP64 pipe issues 1/64 of the FP32 rate, so the per-tile flush stays on the FP32 pipes: the
// 32 lane sums are added by an FP32 shuffle tree (5 roundings on top of the lanes' own FP32 sums) and lane 0 adds
// the warp's tile sum to a compensated (TwoSum, Knuth) hi + lo pair in the same shared slot; the pair becomes an
// FP64 value once, in the block reduction at the end of the kernel.
template <int NV>
struct Partials<float, NV> {
  float t[NV];
  __device__ __forceinline__ Partials() {
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] = 0.f;
  }
  __device__ __forceinline__ void flush(double* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* w2 = reinterpret_cast<float2*>(wsum);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      float v = t[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        float2 acc = w2[warp * NV + j];
        const float s = __fadd_rn(acc.x, v);
        const float bb = __fsub_rn(s, acc.x);
        const float e = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(v, bb));
        acc.x = s;
        acc.y = __fadd_rn(acc.y, e);
        w2[warp * NV + j] = acc;
      }
      t[j] = 0.f;
    }
  }
  __device__ __forceinline__ static double total(const double* wsum, int j) {
    if ((threadIdx.x & 31) != 0) return 0.0;
    const float2 acc = reinterpret_cast<const float2*>(wsum)[(threadIdx.x >> 5) * NV + j];
    return (double)acc.x + (double)acc.y;
  }
};

constexpr int WSUM_MAX = 8;  // warp totals per warp (at least the largest NV of a Partials)

// Block reduction of NV values (bit j of maxmask: value j is a maximum, else a sum) into
// part[bid * NPART + j] (bid: the block's index among the blocks of its reduction, blockIdx.x by
// default); scratch holds at least NTHREADS / 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], unsigned maxmask, double* part, double* scratch,
                                               int bid = -1) {
  if (bid < 0) bid = blockIdx.x;
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
    part[bid * NPART + j] = a;
  }
}

// The same block reduction for values that lane 0 of each warp already holds as the warp's total (the other lanes'
// values are ignored): no shuffle stage, so the FP32 kernels spend only NV short sums of FP64 work here.
template <int NV>
__device__ __forceinline__ void block_partials_warp_totals(const double (&v)[NV], unsigned maxmask, double* part,
                                                           double* scratch, int bid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) scratch[warp * NV + j] = v[j];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double a = scratch[j];
    for (int w = 1; w < NTHREADS / 32; ++w)
      a = ((maxmask >> j) & 1u) ? fmax(a, scratch[w * NV + j]) : a + scratch[w * NV + j];
    part[bid * NPART + j] = a;
  }
}

// Warp maximum of a non-negative FP32 value, at every lane.
__device__ __forceinline__ float warp_max(float m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// True in the block that arrives last of the nblk blocks (gridDim.x by default) counted on ticket;
// that block then sees every block's partials.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket, int nblk = -1) {
  __shared__ int last;
  if (nblk < 0) nblk = gridDim.x;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: totals over all blocks' partials in fixed order; scratch holds NTHREADS * NV doubles.
template <int NV>
__device__ __forceinline__ void total_partials(const double* part, unsigned maxmask, double (&tot)[NV],
                                               double* scratch, int nblk = -1) {
  if (nblk < 0) nblk = gridDim.x;
  double a[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) a[j] = 0.0;  // sums start at 0; maxima are of absolute values
  for (int b = threadIdx.x; b < nblk; b += NTHREADS) {
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

struct Tile {
  int x0, y0, kb, ke;
  bool ee, en;  // the tile also computes the grid's last column (ee) / last row (en), which have no tile
};

__device__ __forceinline__ Tile tile_of(int t, int nx, int ny, int nz, int zcs, int edges) {
  const int nzc = (nz - 2 + zcs - 1) / zcs, ntx = tiles_x(nx, edges);
  const int zc = t % nzc, xy = t / nzc;
  Tile r;
  r.x0 = (xy % ntx) * TX;
  r.y0 = (xy / ntx) * TY;
  r.kb = 1 + zc * zcs;
  r.ke = min(r.kb + zcs, nz - 1);
  r.ee = edge_x(nx, edges) && r.x0 + TX == nx - 1;
  r.en = edge_y(ny, edges) && r.y0 + TY == ny - 1;
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
constexpr int NEDGE = TY + TX + 1;     // edge nodes of a tile at most: last column, last row, corner

// Offsets of a node's four side neighbours in a stencil plane, relative to the node's own slot.
struct Nb {
  int e, w, n, s;
};
__host__ __device__ constexpr Nb nb_tile() { return Nb{1, -1, PW, -PW}; }

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
template <class Op>
__host__ __device__ constexpr int stage_bytes() {
  return (Op::NH + Op::NC) * halo_slot_bytes<typename Op::T>();
}

// bytes of the edge-node records: global index at the tile's first plane, the Ctr of two planes, the face below
template <class Op>
__host__ __device__ constexpr int edge_bytes() {
  return NEDGE * 8 + 2 * NEDGE * (int)sizeof(typename Op::Ctr) + (NEDGE * (int)sizeof(typename Op::T) + 7) / 8 * 8;
}

template <class Op>
__host__ __device__ constexpr int smem_bytes() {
  // stages | three stencil planes | D mbarriers | FP64 warp totals | edge records | 128 bytes of alignment slack
  return Op::D * stage_bytes<Op>() + 3 * PLANE * (int)sizeof(typename Op::T) + Op::D * 8 +
         NTHREADS / 32 * WSUM_MAX * 8 + edge_bytes<Op>() + 128;
}

// The reduction scratch at the end of a kernel reuses the stage ring (all copies consumed by then).
template <class Op>
constexpr bool scratch_fits() {
  return Op::D * stage_bytes<Op>() >= NTHREADS * 8 * (int)sizeof(double);
}

// ------------------------------------------------------------------ face data of a node
// The harmonic face between two nodes from their gh = h^2 / (2 eps): 1 / (gh_a + gh_b) (an approximate FP32
// reciprocal; both nodes of a face form it from the same sum, so the FP32 operator stays symmetric).
__device__ __forceinline__ float gh_face(float ga, float gb) { return __fdividef(1.0f, ga + gb); }

// What centre() reads for a node's faces and output() uses: the stored faces (up from the centre box, east and
// north from the halo box, west and south as the neighbours' east and north faces, or on the first x / y node the
// node's own, which the mirror condition makes equal), or with GH the gh of the node (u) and of its four side
// neighbours (mirror images on the x / y sides), from which output() forms the faces.  PF1's faces are uniform.
template <typename T, bool UNI, bool GH>
struct FaceData {
  T u, e, w, n, s;
  __device__ __forceinline__ void load(T wc, const T* const* H, const T* const* C, int o, bool west, bool south,
                                       bool east, bool north, int iwe, int iwn, int iwu, int igh) {
    if constexpr (UNI) {
      u = e = w = n = s = wc;
    } else if constexpr (GH) {
      const T* gh = H[igh];
      u = gh[o];
      e = gh[east ? o + 1 : o - 1];
      w = gh[west ? o - 1 : o + 1];
      n = gh[north ? o + HBX : o - HBX];
      s = gh[south ? o - HBX : o + HBX];
    } else {
      u = C[iwu][o];
      e = H[iwe][o];
      w = west ? H[iwe][o - 1] : e;
      n = H[iwn][o];
      s = south ? H[iwn][o - HBX] : n;
    }
  }
  // east, west, north and south faces
  __device__ __forceinline__ void sides(T& fe, T& fw, T& fn, T& fs) const {
    if constexpr (GH) {
      fe = gh_face(u, e);
      fw = gh_face(w, u);
      fn = gh_face(u, n);
      fs = gh_face(s, u);
    } else {
      fe = e;
      fw = w;
      fn = n;
      fs = s;
    }
  }
  // the face to the node above, whose face data is hi
  __device__ __forceinline__ T up(T wc, const FaceData& hi) const {
    if constexpr (UNI) {
      return wc;
    } else if constexpr (GH) {
      return gh_face(u, hi.u);
    } else {
      return u;
    }
  }
};

// ------------------------------------------------------------------ the pipelined stencil body
// Op supplies: T, NH, NC, D, CHECK_DONE, Args, Sc, Ctr, Accs and scalars(), q_of(), centre(),
// up_face() (the face between two planes from their Ctr), output() (given the faces below and above),
// finish().  The calling block is block bid of the nblk blocks that share the
// ntiles tiles of one grid (tiles bid, bid + nblk, ...) and its reductions; maps points to the grid's
// tensor maps (kernel parameter or global memory).
// FIXED_ZC: tiles of the compile-time depth ZC (single-grid kernels); else g.zc (batched kernels).
template <class Op, bool FIXED_ZC = true>
__device__ __forceinline__ void stencil_run(const Maps<Op::NH, Op::NC>* __restrict__ maps,
                                            const typename Op::Args& a, const Geom& g, int ntiles, int bid,
                                            int nblk, unsigned long long wait_limit) {
  const int zcs = FIXED_ZC ? ZC : g.zc;
  using T = typename Op::T;
  constexpr int D = Op::D, NH = Op::NH, NC = Op::NC;
  constexpr int HB = halo_slot_bytes<T>(), STAGE = stage_bytes<Op>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // 128-byte aligned start, formed by an offset on the shared array so that the compiler keeps every stage and
  // plane access in the shared address space
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  T* qring = reinterpret_cast<T*>(smem + D * STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + D * STAGE + 3 * PLANE * sizeof(T));
  double* wsum = reinterpret_cast<double*>(bars + D);
  // edge records, each owned by the thread whose halo slot holds the edge node: its global index at the tile's
  // first plane, its Ctr of planes j and j - 1 (between centre() and output()), the face below it
  long* eidx = reinterpret_cast<long*>(wsum + NTHREADS / 32 * WSUM_MAX);
  typename Op::Ctr* ering = reinterpret_cast<typename Op::Ctr*>(eidx + NEDGE);
  T* ewd = reinterpret_cast<T*>(ering + 2 * NEDGE);

  if (Op::CHECK_DONE && *(volatile int*)&a.st->done) return;
  const typename Op::Sc sc = Op::scalars(a);
  if (threadIdx.x == 0) {
    for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
    fence_mbar_init();
  }
  if (threadIdx.x < NTHREADS / 32 * WSUM_MAX) wsum[threadIdx.x] = 0.0;
  __syncthreads();

  // producer (thread 0): the next (tile, plane) of this block's stream of planes
  static_assert((D & (D - 1)) == 0, "the stage ring has a power-of-two size");
  int pt = bid, pj = 0;
  unsigned pseq = 0;
  Tile ptl = tile_of(pt, g.nx, g.ny, g.nz, zcs, g.edges);
  auto issue = [&]() {
    const int stage = pseq & (D - 1);
    unsigned char* sb = smem + stage * STAGE;
    uint64_t* bar = &bars[stage];
    // the centre arrays come as halo boxes when the grid has edge nodes, else as row boxes (no first / last row)
    mbar_expect_tx(bar, (NH * HBY + NC * (g.edges ? HBY : TY)) * HBX * sizeof(T));
    const int k = ptl.kb - 1 + pj;
#pragma unroll
    for (int h = 0; h < NH; ++h) tma_load_3d(sb + h * HB, &maps->h[h], ptl.x0 - 4, ptl.y0 - 1, k, bar);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      tma_load_3d(sb + (NH + c) * HB, &maps->c[c], ptl.x0 - 4, g.edges ? ptl.y0 - 1 : ptl.y0, k, bar);
    ++pseq;
    if (++pj == ptl.ke - ptl.kb + 2) {
      pj = 0;
      pt += nblk;
      if (pt < ntiles) ptl = tile_of(pt, g.nx, g.ny, g.nz, zcs, g.edges);
    }
  };
  if (threadIdx.x == 0)
    for (int d = 0; d < D && pt < ntiles; ++d) issue();

  typename Op::Accs acc;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  unsigned seq = 0;
  bool failed = false;
  for (int t = bid; t < ntiles && !failed; t += nblk) {
    const Tile tl = tile_of(t, g.nx, g.ny, g.nz, zcs, g.edges);
    const TileGeo geo = tile_geo(tl, g.nx, g.ny);
    const int planes = tl.ke - tl.kb + 2;
    // edge role: the node in this thread's halo slot is one of the tile's edge nodes -- the last column (slot
    // es = row), the last row (es = TY + column) or their corner (es = TY + TX).  edge = es | side flags << 6
    // (1 west, 2 south, 4 east, 8 north: the neighbour on that side is a node, not a mirror image), else -1.
    int edge = -1;
    if (geo.hs >= 0 && (tl.ee || tl.en)) {
      int hx, hy;
      halo_pos((int)threadIdx.x - (NTHREADS - NHALO), hx, hy);
      int es = -1;
      if (tl.ee && hx == TX && hy >= 0 && hy < TY && tl.y0 + hy < g.ny) es = hy;
      if (tl.en && hy == TY && hx >= 0 && (hx < TX || tl.ee) && tl.x0 + hx < g.nx) es = TY + hx;
      if (es >= 0) {
        const int gi = tl.x0 + hx, gj = tl.y0 + hy;
        edge = es | ((gi > 0 ? 1 : 0) | (gj > 0 ? 2 : 0) | (gi < g.nx - 1 ? 4 : 0) | (gj < g.ny - 1 ? 8 : 0)) << 6;
        eidx[es] = gi + (long)g.px * gj + g.plane * (tl.kb - 1);
      }
    }
    typename Op::Ctr cprev{}, cnow{};
    T q_dn = T(0), q_prev = T(0), wD = T(0);
    // offsets of the three stencil planes in the ring (integers, so that every access stays a shared-memory
    // access of the ring): plane j, plane j - 1, plane j - 2 (free for plane j + 1)
    int qnow = 0, qprev = 2 * PLANE, qold = PLANE;
    long cidx = geo.gi + (long)g.px * geo.gj + g.plane * (tl.kb - 1);
    // Op::UNROLL = 2: the two Ctr values trade roles without copies (where registers allow)
#pragma unroll(Op::UNROLL)
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
        // a row box lacks the halo box's first row: shift its base so that both are indexed by halo-box offsets
        const int crow = g.edges ? 0 : HBX * (int)sizeof(T);
#pragma unroll
        for (int c = 0; c < NC; ++c) C[c] = reinterpret_cast<const T*>(sb + (NH + c) * HB - crow);
        if (edge >= 0) {  // the edge node's stencil value and its Ctr of plane j, written straight to shared memory
          typename Op::Ctr& ce = ering[(j & 1) * NEDGE + (edge & 63)];
          qring[qnow + geo.hs] = Op::q_of(sc, H, geo.hbo, &ce);
          Op::centre(sc, a, H, C, geo.hbo, (edge >> 6) & 1, (edge >> 7) & 1, (edge >> 8) & 1, (edge >> 9) & 1, ce);
        }
        if (geo.cbo >= 0) qc = Op::q_of(sc, H, geo.cbo, &cnow);
        if (geo.valid)
          Op::centre(sc, a, H, C, geo.cbo, geo.gi > 0, geo.gj > 0, geo.gi < g.nx - 1, geo.gj < g.ny - 1, cnow);
        qring[qnow + cs(lx, ly)] = qc;
        if (geo.hs >= 0 && edge < 0) qring[qnow + geo.hs] = geo.hbo >= 0 ? Op::q_of(sc, H, geo.hbo, nullptr) : T(0);
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
      if (j >= 1) {
        const T wUp = Op::up_face(a, cprev, cnow);  // the face between planes j - 1 and j
        if (j >= 2 && geo.valid)
          Op::output(sc, a, qring + qprev, cs(lx, ly), nb_tile(), cidx, cprev, q_dn, qc, wD, wUp, acc);
        q_dn = q_prev;
        wD = wUp;
        cidx += g.plane;
        if (edge >= 0) {  // the edge node of plane j - 1: its stencil values below and above are in the ring
          const int es = edge & 63;
          const typename Op::Ctr& ep = ering[((j - 1) & 1) * NEDGE + es];
          const T wUe = Op::up_face(a, ep, ering[(j & 1) * NEDGE + es]);
          if (j >= 2) {
            // a side neighbour beyond the last column / row is the mirror image of the one before it
            const Nb nbe{(edge >> 8) & 1 ? 1 : -1, -1, (edge >> 9) & 1 ? PW : -PW, -PW};
            Op::output(sc, a, qring + qprev, geo.hs, nbe, eidx[es] + g.plane * (j - 1), ep, qring[qold + geo.hs],
                       qring[qnow + geo.hs], ewd[es], wUe, acc);
          }
          ewd[es] = wUe;
        }
      }
      q_prev = qc;
      cprev = cnow;
      // rotate the three stencil planes
      const int freed = qold;
      qold = qprev;
      qprev = qnow;
      qnow = freed;
    }
    acc.flush(wsum);
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
  Op::finish(a, acc, wsum, reinterpret_cast<double*>(smem), bid, nblk);
}

// ------------------------------------------------------------------ phase B: s = r - alpha v, t = A M^-1 s
template <typename T_, bool UNI>
struct OpB {
  using T = T_;
  static constexpr bool GH = false;
  static constexpr int NH = SlotsB<T_, UNI>::NH, NC = SlotsB<T_, UNI>::NC, D = sizeof(T_) == 4 ? 4 : 2;
  static constexpr int MINB = sizeof(T_) == 4 ? 4 : 2;
  static constexpr int UNROLL = 2;
  static constexpr bool CHECK_DONE = true;
  enum { R = 0, V = 1, DI = 2, WE = 3, WN = 4, GHS = 0 };
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
    T s, di, rt;
    FaceData<T, UNI, GH> f;
  };
  struct Accs {
    Partials<T, 5> p;  // r~.s, r~.t, t.s, t.t, s.s
    T smax = T(0);
    __device__ void flush(double* wsum) { p.flush(wsum); }
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
  __device__ static void centre(const Sc&, const Args& a, const T* const* H, const T* const* C, int o, bool west,
                                bool south, bool east, bool north, Ctr& c) {
    c.rt = C[RT][o];
    c.f.load(a.wc, H, C, o, west, south, east, north, WE, WN, WU, GHS);
  }
  __device__ static T up_face(const Args& a, const Ctr& lo, const Ctr& hi) { return lo.f.up(a.wc, hi.f); }
  __device__ static void output(const Sc&, const Args& a, const T* Q, int pc, Nb nb, long cidx, const Ctr& c, T q_dn,
                                T q_up, T wD, T wU, Accs& acc) {
    T tc;
    if (c.di == T(0)) {
      tc = c.s;
    } else {
      const T qE = Q[pc + nb.e], qW = Q[pc + nb.w], qN = Q[pc + nb.n], qS = Q[pc + nb.s];
      T nb;
      if (UNI) {
        nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        T fe, fw, fn, fs;
        c.f.sides(fe, fw, fn, fs);
        nb = fe * qE;
        nb = fma(fw, qW, nb);
        nb = fma(fn, qN, nb);
        nb = fma(fs, qS, nb);
        nb = fma(wU, q_up, nb);
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
  __device__ static void finish(const Args& a, const Accs& acc, const double* wsum, double* scratch, int bid,
                                int nblk) {
    using P = Partials<T, 5>;
    if constexpr (sizeof(T) == 4) {
      const double vals[6] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), P::total(wsum, 3),
                              P::total(wsum, 4), (double)warp_max(acc.smax)};
      block_partials_warp_totals<6>(vals, 32u, a.part, scratch, bid);
    } else {
      double vals[6] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), P::total(wsum, 3),
                        P::total(wsum, 4), (double)acc.smax};
      block_partials<6>(vals, 32u, a.part, scratch, bid);
    }
    if (!arrive_last(&a.st->ticket, nblk)) return;
    double tot[6];
    total_partials<6>(a.part, 32u, tot, scratch, nblk);
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
  static constexpr bool GH = !UNI && ca_face_from_gh<T_>();
  static constexpr int NH = SlotsCA<T_, UNI>::NH, NC = SlotsCA<T_, UNI>::NC, D = 2;
  static constexpr int MINB = sizeof(T_) == 4 ? 4 : 2;
  static constexpr int UNROLL = UNI ? 2 : 1;
  static constexpr bool CHECK_DONE = true;
  enum { R = 0, V = 1, TT = 2, P = 3, DI = 4, WE = 5, WN = 6, GHS = 5 };
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
    T s, rn, pn, pold, di, x, rt;
    FaceData<T, UNI, GH> f;
  };
  struct Accs {
    Partials<T, 3> p;  // r~.v', r~.r', r'.r'
    T rmax = T(0);
    __device__ void flush(double* wsum) { p.flush(wsum); }
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
  __device__ static void centre(const Sc&, const Args& a, const T* const* H, const T* const* C, int o, bool west,
                                bool south, bool east, bool north, Ctr& c) {
    c.x = C[X][o];
    c.rt = C[RT][o];
    c.f.load(a.wc, H, C, o, west, south, east, north, WE, WN, WU, GHS);
  }
  __device__ static T up_face(const Args& a, const Ctr& lo, const Ctr& hi) { return lo.f.up(a.wc, hi.f); }
  __device__ static void output(const Sc& sc, const Args& a, const T* Q, int pc, Nb nb, long cidx, const Ctr& c,
                                T q_dn, T q_up, T wD, T wU, Accs& acc) {
    T vn;
    if (c.di == T(0)) {
      vn = c.pn;
    } else {
      const T qE = Q[pc + nb.e], qW = Q[pc + nb.w], qN = Q[pc + nb.n], qS = Q[pc + nb.s];
      T nb;
      if (UNI) {
        nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        T fe, fw, fn, fs;
        c.f.sides(fe, fw, fn, fs);
        nb = fe * qE;
        nb = fma(fw, qW, nb);
        nb = fma(fn, qN, nb);
        nb = fma(fs, qS, nb);
        nb = fma(wU, q_up, nb);
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
  __device__ static void finish(const Args& a, const Accs& acc, const double* wsum, double* scratch, int bid,
                                int nblk) {
    using P = Partials<T, 3>;
    if constexpr (sizeof(T) == 4) {
      const double vals[4] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), (double)warp_max(acc.rmax)};
      block_partials_warp_totals<4>(vals, 8u, a.part, scratch, bid);
    } else {
      double vals[4] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), (double)acc.rmax};
      block_partials<4>(vals, 8u, a.part, scratch, bid);
    }
    if (!arrive_last(&a.st->ticket, nblk)) return;
    double tot[4];
    total_partials<4>(a.part, 8u, tot, scratch, nblk);
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

// ------------------------------------------------------------------ conjugate gradients, one pass per iteration
// Jacobi-preconditioned CG for the symmetric systems (Section 3: Eq. 9 and PF1; with zero-jump faces PF2 too) in
// the single-reduction form of Chronopoulos and Gear, in the inner product <u, v>_w = sum_c w_c u_c v_c that weights
// a node by 1/2 for every x or y side it lies on (A is symmetric in it; see pf_cg.cu).  With z = M^-1 r, w = A z,
// s = A p, gamma = <r, z>_w, delta = <w, z>_w, one pass of iteration i forms at every node
//   s_i = w_i + beta_i s_{i-1},  r_{i+1} = r_i - alpha_i s_i,  z_{i+1} = M^-1 r_{i+1},
//   p_i = z_i + beta_i p_{i-1},  x_{i+1} = x_i + alpha_i p_i,    w_{i+1} = A z_{i+1} (the stencil),
// and gamma_{i+1}, delta_{i+1}; the last block sets beta_{i+1} = gamma_{i+1} / gamma_i and
// alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i).  The prime pass (alpha = beta = 0
// on zeroed w, s, p) gives w_0 = A z_0, alpha_0 = gamma_0 / delta_0.  On identity rows r, w, s and p vanish.
template <typename T_, bool UNI>
struct OpCG {
  using T = T_;
  static constexpr bool GH = !UNI && ca_face_from_gh<T_>();
  static constexpr int NH = SlotsCG<T_, UNI>::NH, NC = SlotsCG<T_, UNI>::NC, D = 2;
  static constexpr int MINB = sizeof(T_) == 4 ? 4 : 2;
  static constexpr int UNROLL = 1;
  static constexpr bool CHECK_DONE = true;
  enum { R = 0, W = 1, S = 2, DI = 3, WE = 4, WN = 5, GHS = 4 };
  enum { P = 0, X = 1, WU = 2 };
  struct Args {
    double* part;
    BicgState* st;
    T* r_out;
    T* w_out;
    T* s_out;
    T* p;  // p_{i-1} in, p_i out (read at the node only)
    T* x;
    T wc;
    int prime;
  };
  struct Sc {
    T al, be;
  };
  struct Ctr {
    T s, rn, zold, pn, xn, di, sw;
    FaceData<T, UNI, GH> f;
  };
  struct Accs {
    Partials<T, 3> p;  // gamma' = <r', z'>_w, delta' = <w', z'>_w, r'.r'
    T rmax = T(0);
    __device__ void flush(double* wsum) { p.flush(wsum); }
  };
  __device__ static Sc scalars(const Args& a) { return Sc{(T)a.st->alpha, (T)a.st->beta}; }
  __device__ static T q_of(const Sc& sc, const T* const* H, int o, Ctr* c) {
    const T s = fma(sc.be, H[S][o], H[W][o]);
    const T r = H[R][o];
    const T rn = fma(-sc.al, s, r);
    const T di = H[DI][o];
    if (c) {
      c->s = s;
      c->rn = rn;
      c->zold = di * r;
      c->di = di;
    }
    return di * rn;  // z_{i+1}, the stencil's input
  }
  __device__ static void centre(const Sc& sc, const Args& a, const T* const* H, const T* const* C, int o, bool west,
                                bool south, bool east, bool north, Ctr& c) {
    c.pn = fma(sc.be, C[P][o], c.zold);
    c.xn = fma(sc.al, c.pn, C[X][o]);
    c.sw = (west && east ? T(1) : T(0.5)) * (south && north ? T(1) : T(0.5));
    c.f.load(a.wc, H, C, o, west, south, east, north, WE, WN, WU, GHS);
  }
  __device__ static T up_face(const Args& a, const Ctr& lo, const Ctr& hi) { return lo.f.up(a.wc, hi.f); }
  __device__ static void output(const Sc&, const Args& a, const T* Q, int pc, Nb nb, long cidx, const Ctr& c, T q_dn,
                                T q_up, T wD, T wU, Accs& acc) {
    T wn;
    if (c.di == T(0)) {
      wn = c.rn;
    } else {
      const T qE = Q[pc + nb.e], qW = Q[pc + nb.w], qN = Q[pc + nb.n], qS = Q[pc + nb.s];
      T nbs;
      if (UNI) {
        nbs = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
      } else {
        T fe, fw, fn, fs;
        c.f.sides(fe, fw, fn, fs);
        nbs = fe * qE;
        nbs = fma(fw, qW, nbs);
        nbs = fma(fn, qN, nbs);
        nbs = fma(fs, qS, nbs);
        nbs = fma(wU, q_up, nbs);
        nbs = fma(wD, q_dn, nbs);
      }
      wn = c.rn - nbs;
      if (!a.prime) a.x[cidx] = c.xn;
    }
    a.r_out[cidx] = c.rn;
    a.w_out[cidx] = wn;
    a.s_out[cidx] = c.s;
    a.p[cidx] = c.pn;
    const T z = c.di * c.rn, swz = c.sw * z;
    acc.p.t[0] = fma(swz, c.rn, acc.p.t[0]);
    acc.p.t[1] = fma(swz, wn, acc.p.t[1]);
    acc.p.t[2] = fma(c.rn, c.rn, acc.p.t[2]);
    acc.rmax = fmax(acc.rmax, tabs(c.rn));
  }
  __device__ static void finish(const Args& a, const Accs& acc, const double* wsum, double* scratch, int bid,
                                int nblk) {
    using P = Partials<T, 3>;
    if constexpr (sizeof(T) == 4) {
      const double vals[4] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), (double)warp_max(acc.rmax)};
      block_partials_warp_totals<4>(vals, 8u, a.part, scratch, bid);
    } else {
      double vals[4] = {P::total(wsum, 0), P::total(wsum, 1), P::total(wsum, 2), (double)acc.rmax};
      block_partials<4>(vals, 8u, a.part, scratch, bid);
    }
    if (!arrive_last(&a.st->ticket, nblk)) return;
    double tot[4];
    total_partials<4>(a.part, 8u, tot, scratch, nblk);
    if (threadIdx.x != 0) return;
    BicgState* st = a.st;
    const double ga = tot[0], de = tot[1], r2 = tot[2], rmx = tot[3];
    st->ticket = 0;
    if (!a.prime) {
      st->iter += 1;
      st->rnorm2 = r2;
      st->rinf = rmx;
      const bool conv = st->norm == 0 ? (r2 <= st->tol2) : (rmx < st->tol);
      if (conv) {
        st->done = 1;
        st->status = 0;
        return;
      }
      if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = 3;  // PF_E_NOCONV
        return;
      }
    }
    // gamma and delta are positive for a positive definite operator on a non-zero residual
    double al = 0.0, be = 0.0;
    if (a.prime || st->alpha == 0.0) {
      al = ga / de;
    } else {
      be = ga / st->rho;
      al = ga / (de - be * ga / st->alpha);
    }
    if (!(ga > 0.0) || !(de > 0.0) || !(al > 0.0) || !isfinite(al) || !isfinite(be)) {
      st->done = 1;
      st->status = 4;  // PF_E_BREAKDOWN
      return;
    }
    st->rho = ga;
    st->alpha = al;
    st->beta = be;
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
  static constexpr int MINB = 3;  // 24 warps per SM hide the FP64 pipe's latency better than 16
  static constexpr int UNROLL = UNI ? 2 : 1;
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
    int need_bb = 1;   // 0: b.b of this right-hand side is already in st->bnorm2 (later refinement steps)
    int need_max = 1;  // 0: the stop test is the 2-norm, max |r| is not needed
    // init = 0 with in_r set: start the FP32 inner solve of refinement here (in place of writing r32 and a
    // separate start kernel): r = r~ = (float) r, p = v = t = d = 0, and its state st2 from ||r||^2
    float *in_r = nullptr, *in_rt = nullptr, *in_p = nullptr, *in_v = nullptr, *in_t = nullptr, *in_d = nullptr;
    BicgState* st2 = nullptr;
  };
  struct Sc {
    int unused;
  };
  struct Ctr {
    double b, diag;
    bool ident;  // an identity row (Jacobi scaling +0); x at the node is the stencil plane's centre value
    FaceData<double, UNI, false> f;
  };
  struct Accs {
    double rr = 0.0, bb = 0.0, rmax = 0.0;
    __device__ void flush(double*) {}
  };
  __device__ static Sc scalars(const Args&) { return Sc{0}; }
  __device__ static double q_of(const Sc&, const double* const* H, int o, Ctr* c) {
    const double xv = H[X][o];
    if (c) c->ident = __double_as_longlong(H[DI][o]) == 0;
    return xv;
  }
  __device__ static void centre(const Sc&, const Args& a, const double* const* H, const double* const* C, int o,
                                bool west, bool south, bool east, bool north, Ctr& c) {
    c.b = C[B][o];
    if constexpr (UNI) {
      c.diag = a.diagc;
    } else {
      c.diag = C[DG][o];
    }
    c.f.load(a.wc, H, C, o, west, south, east, north, WE, WN, WU, 0);
  }
  __device__ static double up_face(const Args& a, const Ctr& lo, const Ctr& hi) { return lo.f.up(a.wc, hi.f); }
  __device__ static void output(const Sc&, const Args& a, const double* Q, int pc, Nb nb, long cidx, const Ctr& c,
                                double q_dn, double q_up, double wD, double wU, Accs& acc) {
    double rc;
    const double xc = Q[pc];
    if (c.ident) {
      rc = c.b - xc;
    } else {
      const double qE = Q[pc + nb.e], qW = Q[pc + nb.w], qN = Q[pc + nb.n], qS = Q[pc + nb.s];
      if (UNI) {
        const double nb = a.wc * (((qE + qW) + (qN + qS)) + (q_up + q_dn));
        rc = c.b - (c.diag * xc - nb);
      } else {
        // b + sum of face * neighbour, then - diag * x: seven FP64 operations
        double fe, fw, fn, fs;
        c.f.sides(fe, fw, fn, fs);
        double acc_b = fma(fe, qE, c.b);
        acc_b = fma(fw, qW, acc_b);
        acc_b = fma(fn, qN, acc_b);
        acc_b = fma(fs, qS, acc_b);
        acc_b = fma(wU, q_up, acc_b);
        acc_b = fma(wD, q_dn, acc_b);
        rc = fma(-c.diag, xc, acc_b);
      }
    }
    if (a.init) {
      a.r[cidx] = rc;
      a.rt[cidx] = rc;
      a.p[cidx] = 0.0;
      a.v[cidx] = 0.0;
      a.t[cidx] = 0.0;
    } else if (a.in_r) {
      const float rf = (float)rc;
      a.in_r[cidx] = rf;
      a.in_rt[cidx] = rf;
      a.in_p[cidx] = 0.f;
      a.in_v[cidx] = 0.f;
      a.in_t[cidx] = 0.f;
      a.in_d[cidx] = 0.f;
    } else {
      a.r32[cidx] = (float)rc;
    }
    acc.rr = fma(rc, rc, acc.rr);
    if (a.need_bb) acc.bb = fma(c.b, c.b, acc.bb);
    if (a.need_max) acc.rmax = fmax(acc.rmax, fabs(rc));
  }
  __device__ static void finish(const Args& a, const Accs& acc, const double* wsum, double* scratch, int bid,
                                int nblk) {
    double vals[3] = {acc.rr, acc.bb, acc.rmax};
    block_partials<3>(vals, 4u, a.part, scratch, bid);
    if (!arrive_last(&a.st->ticket, nblk)) return;
    double tot[3];
    total_partials<3>(a.part, 4u, tot, scratch, nblk);
    if (threadIdx.x != 0) return;
    BicgState* st = a.st;
    // bnorm2 was preset to b.b over the Dirichlet planes, or kept from the first residual of this solve
    double bb = a.need_bb ? tot[1] + st->bnorm2 : st->bnorm2;
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
    if (a.st2) {  // the FP32 inner solve on r starts here (its tolerance, norm and limit were set before)
      BicgState* s2 = a.st2;
      const double b2 = tot[0] > 0.0 ? tot[0] : 1.0;
      s2->bnorm2 = b2;
      s2->rho = tot[0];
      s2->rnorm2 = tot[0];
      s2->rinf = tot[2];
      set_tol2(s2, tot[0], b2);
      s2->alpha = s2->omega = s2->beta = 0.0;
      s2->sexit = 0;
      s2->iter = 0;
      s2->status = 0;
      s2->done = (s2->norm == 0 ? tot[0] <= s2->tol2 : tot[2] < s2->tol) ? 1 : 0;
      s2->ticket = 0;
    }
  }
};

}  // namespace pf
