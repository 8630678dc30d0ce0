// pf_batch.cu -- many independent PF problems solved together: the batched engine behind pf_batch_* and
// the server.  Every BiCGSTAB phase (Table 3) and every FP64 residual of all problems that need one at the
// same time runs as ONE launch of a batched stencil kernel, and each problem's chunk of BiCGSTAB iterations
// between host checks is part of a captured CUDA graph that all iterating problems share.
//
// Scheduling is per problem (iteration-level): every problem is a state machine (operators, initial
// potential, Fermi step, PF1 solve, PF2 solve, outer update, outputs; inside a linear solve: FP64 residual,
// FP32 inner start, inner chunks, or the FP64 chunks), and every engine tick advances each problem by one
// step.  The launches of a tick are shared by the problems whose step needs them, so a problem never waits
// for another problem's linear solve to finish, and problems can join or leave between ticks.
//
// The batched kernel gives each problem a contiguous range of blocks: nblk = ceil(ntiles / tiles_per_block)
// blocks, so a block works for one problem only and reduces into that problem's partials and state exactly
// as the single-grid kernel does.  A problem's arithmetic and reduction order therefore depend only on its
// own size and tiles_per_block: its result is bitwise the same alone or in any mix.  A per-launch block map
// (rewritten every tick) sends the blocks of problems that do not take part in that launch home at once.
// tiles_per_block is chosen by timing the FP32 phase kernels of the batch's own operators for each
// candidate (pf_batch_autotune), or set by the caller.  The tensor maps and arguments of all problems live
// in device tables that each block reads at start.
#include <chrono>

#include "pf_decomp.cuh"
#include "pf_grid.cuh"
#include "pf_stencil.cuh"

namespace pf {

template <class Op>
struct alignas(64) BatchItem {
  Maps<Op::NH, Op::NC> maps;
  typename Op::Args a;
  Geom g;
  int ntiles, block0, nblk;
};

// the FP64 residual, skipping grids whose state is already done
template <bool UNI>
struct OpResSkip : OpRes<UNI> {
  static constexpr bool CHECK_DONE = true;
};

// A tensor map in global memory is read through the tensormap proxy: order it after the generic-proxy
// writes that placed it there.
__device__ __forceinline__ void tensormap_acquire(const void* p) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(p) : "memory");
}

// Block b works for problem block_item[b].x as its block block_item[b].y (of the problem's nblk); a map lists
// only the blocks of the problems that take part in the launch.
template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB)
    k_stencil_batch(const BatchItem<Op>* __restrict__ items, const int2* __restrict__ block_item,
                    unsigned long long wait_limit) {
  const int2 e = block_item[blockIdx.x];
  if (e.x < 0) return;
  const BatchItem<Op>* it = items + e.x;
  __shared__ typename Op::Args sa;
  __shared__ Geom sg;
  __shared__ int sn[3];
  if (threadIdx.x == 0) {
    sa = it->a;
    sg = it->g;
    sn[0] = it->ntiles;
    sn[1] = e.y;
    sn[2] = it->nblk;
#pragma unroll
    for (int h = 0; h < Op::NH; ++h) tensormap_acquire(&it->maps.h[h]);
#pragma unroll
    for (int c = 0; c < Op::NC; ++c) tensormap_acquire(&it->maps.c[c]);
  }
  __syncthreads();
  stencil_run<Op, false>(&it->maps, sa, sg, sn[0], sn[1], sn[2], wait_limit);
}

// dst[i] = *st64[i] (FP64 / refinement state) and dst[n + i] = *st32[i] (FP32 inner state) of every member
__global__ void k_gather_states(BicgState* const* __restrict__ st64, BicgState* const* __restrict__ st32, int n,
                                BicgState* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    dst[i] = *st64[i];
    dst[n + i] = *st32[i];
  }
}

}  // namespace pf

using namespace pfi;
using pf::BicgState;

using namespace pfi;
using pf::BicgState;

namespace {

// the launch kinds of a tick, per operator (x3): map slots in the device map pool
enum { K_RES0 = 0, K_RES1, K_PRIME32, K_PRIME64, K_CHUNK32, K_CHUNK64, K_PER_OP };
constexpr int N_OPS = 3;
constexpr int SLOT_FULL = N_OPS * K_PER_OP;  // every member active (autotuner)
constexpr int N_SLOTS = SLOT_FULL + 1;

}  // namespace

struct pf_batch {
  std::vector<pf_grid*> grids;    // grids[i] belongs to members[i]
  std::vector<pfi::BatchMember> members;
  cudaStream_t user = nullptr;    // the caller's stream
  cudaStream_t stream = nullptr;  // the batch's own stream: per-problem work, tables, state read-back
  cudaStream_t ops[N_OPS] = {};   // the batched launches of each operator run concurrently on these
  cudaStream_t cstream = nullptr; // chunk graphs are captured here
  cudaEvent_t fork = nullptr, join[N_OPS] = {};
  cudaEvent_t tick0 = nullptr, tick1 = nullptr;  // device span of a tick's work (launches to state read-back)
  pf_batch_stats stats{};                        // of the last pf_batch_nonlinear_solve
  int tpb = 0;                    // tiles per block; 0: tune at the next solve
  int zc = pf::ZC;                // interior z-planes per tile
  pf_batch_tune tune{};
  // device arena for launch tables, filled from a pinned staging copy
  unsigned char* darena = nullptr;
  unsigned char* harena = nullptr;
  size_t cap = 0, top = 0;
  // tables built for the current membership (invalidated when it changes)
  bool built = false;
  int nblocks = 0;                      // blocks of all members together
  std::vector<int> block0, nblk, ntl;   // block range and tile count of each member
  int2* dmaps = nullptr;                // N_SLOTS block maps of up to nblocks entries
  std::vector<int2> hmaps;
  int mapn[N_SLOTS] = {};               // entries of each map in this tick (the launch's grid size)
  BicgState** dst64 = nullptr;          // members' state pointers (device)
  BicgState** dst32 = nullptr;
  std::map<std::string, const void*> items;
  // chunk graphs: the instantiated graph, its kernel nodes, and the grid size they were last given
  struct Chunk {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;
    int grid = 0;
  };
  std::map<std::string, Chunk> graphs;
  BicgState* dgather = nullptr;         // gathered states (device) and their pinned copy
  BicgState* hgather = nullptr;
  int gather_cap = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

constexpr size_t ARENA_BYTES = 16u << 20;
// BiCGSTAB iterations per engine tick (even: every chunk starts at ping-pong parity 1); a problem whose
// solve ends inside a chunk skips the rest of it (its state is done)
constexpr int TICK_ITERS = 4;
const int TPB_CANDIDATES[] = {1, 2, 4, 8, 16};
const int ZC_CANDIDATES[] = {16, 32, 64};

template <typename T>
OpArrays<T> opsT(const pf_grid* g, int op);
template <>
OpArrays<double> opsT<double>(const pf_grid* g, int op) { return ops64(g, op); }
template <>
OpArrays<float> opsT<float>(const pf_grid* g, int op) { return ops32(g, op); }
template <typename T>
Krylov<T> kryT(pf_grid* g);
template <>
Krylov<double> kryT<double>(pf_grid* g) { return kry64(g); }
template <>
Krylov<float> kryT<float>(pf_grid* g) { return kry32(g); }

int blocks_for(int ntiles, int tpb) {
  int b = (ntiles + tpb - 1) / tpb;
  const int cap = pf::max_partial_blocks();
  if (b > cap) b = cap;
  if (b > ntiles) b = ntiles;
  return b < 1 ? 1 : b;
}

void drain(pf_batch* B) {
  cudaStreamSynchronize(B->stream);
  for (int o = 0; o < N_OPS; ++o)
    if (B->ops[o]) cudaStreamSynchronize(B->ops[o]);
}

// Forgets every table and graph (after every stream drained).
void invalidate(pf_batch* B) {
  drain(B);
  for (auto& kv : B->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  B->graphs.clear();
  B->items.clear();
  B->top = 0;
  B->built = false;
}

// Copies host bytes into the arena and waits for the copy, so that launches on any stream may read them;
// nullptr when the arena is full.
const void* upload(pf_batch* B, const void* src, size_t bytes) {
  const size_t at = (B->top + 255) / 256 * 256;
  if (at + bytes > B->cap) return nullptr;
  cudaStreamSynchronize(B->stream);
  memcpy(B->harena + at, src, bytes);
  if (cudaMemcpyAsync(B->darena + at, B->harena + at, bytes, cudaMemcpyHostToDevice, B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess)
    return nullptr;
  B->top = at + bytes;
  return B->darena + at;
}

// Block ranges, map pool and state pointers for the current members (tables are built on first use).
pf_status build(pf_batch* B) {
  if (B->built) return PF_OK;
  invalidate(B);
  const int n = (int)B->grids.size();
  B->block0.assign(n, 0);
  B->nblk.assign(n, 0);
  B->ntl.assign(n, 0);
  int nb = 0;
  for (int i = 0; i < n; ++i) {
    const pf_grid* g = B->grids[i];
    B->ntl[i] = pf::tiles_for(g->nx, g->ny, g->nz, B->zc, 1);
    B->block0[i] = nb;
    B->nblk[i] = blocks_for(B->ntl[i], B->tpb);
    nb += B->nblk[i];
  }
  B->nblocks = nb;
  B->hmaps.assign((size_t)N_SLOTS * nb, make_int2(-1, 0));
  for (int i = 0; i < n; ++i)
    for (int b = 0; b < B->nblk[i]; ++b) B->hmaps[(size_t)SLOT_FULL * nb + B->block0[i] + b] = make_int2(i, b);
  B->mapn[SLOT_FULL] = nb;
  B->dmaps = (int2*)upload(B, B->hmaps.data(), B->hmaps.size() * sizeof(int2));
  std::vector<BicgState*> s64, s32;
  for (pf_grid* g : B->grids) {
    s64.push_back(g->st);
    s32.push_back(g->st2);
  }
  B->dst64 = (BicgState**)upload(B, s64.data(), s64.size() * sizeof(BicgState*));
  B->dst32 = (BicgState**)upload(B, s32.data(), s32.size() * sizeof(BicgState*));
  if (!B->dmaps || !B->dst64 || !B->dst32) return fail(PF_E_OOM, "batch launch tables do not fit");
  if (n > B->gather_cap) {
    if (B->dgather) cudaFree(B->dgather);
    if (B->hgather) cudaFreeHost(B->hgather);
    B->dgather = nullptr;
    B->hgather = nullptr;
    B->gather_cap = 0;
    PF_CK(cudaMalloc(&B->dgather, 2 * n * sizeof(BicgState)));
    PF_CK(cudaMallocHost(&B->hgather, 2 * n * sizeof(BicgState)));
    B->gather_cap = n;
  }
  B->built = true;
  return PF_OK;
}

const int2* map_of(pf_batch* B, int slot) { return B->dmaps + (size_t)slot * B->nblocks; }

// The item table of one launch kind over all members, built on first use.
template <class Op, class Fill>
pf_status items_for(pf_batch* B, const std::string& key, Fill fill, const void** out) {
  auto it = B->items.find(key);
  if (it != B->items.end()) {
    *out = it->second;
    return PF_OK;
  }
  std::vector<pf::BatchItem<Op>> v(B->grids.size());
  for (size_t j = 0; j < B->grids.size(); ++j) {
    pf_grid* g = B->grids[j];
    PF_TRY(fill((int)j, g, v[j]));
    v[j].g = g->geom;
    v[j].g.zc = B->zc;
    v[j].g.edges = 1;  // a batch launch holds many tiles per block
    v[j].ntiles = B->ntl[j];
    v[j].nblk = B->nblk[j];
    v[j].block0 = B->block0[j];
  }
  const void* d = upload(B, v.data(), v.size() * sizeof(v[0]));
  if (!d) return fail(PF_E_OOM, "batch launch tables do not fit");
  B->items[key] = d;
  *out = d;
  return PF_OK;
}

template <class Op>
pf_status launch_items(pf_batch* B, const void* items, const int2* map, int grid, cudaStream_t st) {
  static_assert(pf::scratch_fits<Op>(), "reduction scratch must fit in the stage ring");
  if (grid < 1) return PF_OK;
  pf::k_stencil_batch<Op><<<grid, pf::NTHREADS, pf::smem_bytes<Op>(), st>>>(
      static_cast<const pf::BatchItem<Op>*>(items), map, WAIT_LIMIT);
  PF_CK(cudaGetLastError());
  return PF_OK;
}

template <class Op>
void set_smem_attr() {
  cudaFuncSetAttribute(pf::k_stencil_batch<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf::smem_bytes<Op>());
  cudaFuncSetAttribute(pf::k_stencil_batch<Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

template <typename T, bool UNI>
void set_attrs() {
  set_smem_attr<pf::OpB<T, UNI>>();
  set_smem_attr<pf::OpCA<T, UNI>>();
  if constexpr (sizeof(T) == 8) set_smem_attr<pf::OpResSkip<UNI>>();
}

std::string key_of(const char* kind, int op, int f64, int par) {
  char buf[64];
  snprintf(buf, sizeof buf, "%s|%d|%d|%d", kind, op, f64, par);
  return buf;
}

// The unknown and right-hand side of each operator's linear solve inside the nonlinear iteration.
double* x_of(pf_grid* g, int op) { return op == PF_OP_POISSON ? g->phi0 : op == PF_OP_PF1 ? g->psi : g->phi; }
const double* b_of(const pf_grid* g, int op) { return op == PF_OP_PF1 ? g->b1 : g->b2; }

// ---- item fillers (the same arrays, in the same slots, as the single-grid launches)
template <typename T, bool UNI>
pf_status fill_b(pf_grid* g, int op, int cur, pf::BatchItem<pf::OpB<T, UNI>>& it) {
  using SB = pf::SlotsB<T, UNI>;
  const OpArrays<T> A = opsT<T>(g, op);
  const Krylov<T> K = kryT<T>(g);
  if constexpr (UNI) {
    const T* h[SB::NH] = {K.r[cur], K.v[cur], A.dinv};
    const T* c[SB::NC] = {K.rt};
    PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &it.maps, h, c, 1)));
  } else {
    const T* h[SB::NH] = {K.r[cur], K.v[cur], A.dinv, A.wE, A.wN};
    const T* c[SB::NC] = {K.rt, A.wU};
    PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &it.maps, h, c, 1)));
  }
  it.a = typename pf::OpB<T, UNI>::Args{g->part, sizeof(T) == 8 ? g->st : g->st2, K.t, (T)A.wc};
  return PF_OK;
}

template <typename T, bool UNI>
pf_status fill_ca(pf_grid* g, int op, int cur, int prime, T* x, pf::BatchItem<pf::OpCA<T, UNI>>& it) {
  using SC = pf::SlotsCA<T, UNI>;
  const OpArrays<T> A = opsT<T>(g, op);
  const Krylov<T> K = kryT<T>(g);
  if constexpr (UNI) {
    const T* h[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv};
    const T* c[SC::NC] = {x, K.rt};
    PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &it.maps, h, c, 1)));
  } else if constexpr (pf::ca_face_from_gh<T>()) {
    const T* h[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv, A.gh};
    const T* c[SC::NC] = {x, K.rt};
    PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &it.maps, h, c, 1)));
  } else {
    const T* h[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv, A.wE, A.wN};
    const T* c[SC::NC] = {x, K.rt, A.wU};
    PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &it.maps, h, c, 1)));
  }
  it.a = typename pf::OpCA<T, UNI>::Args{g->part, sizeof(T) == 8 ? g->st : g->st2, x, K.r[1 - cur], K.p[1 - cur],
                                         K.v[1 - cur], (T)A.wc, prime};
  return PF_OK;
}

template <bool UNI>
pf_status fill_res(pf_grid* g, int op, int init, const double* x, const double* b,
                   pf::BatchItem<pf::OpResSkip<UNI>>& it) {
  using S = pf::SlotsRes<UNI>;
  const OpArrays<double> A = ops64(g, op);
  const Krylov<double> K = kry64(g);
  if constexpr (UNI) {
    const double* h[S::NH] = {x, A.dinv};
    const double* c[S::NC] = {b};
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &it.maps, h, c, 1)));
  } else {
    const double* h[S::NH] = {x, A.dinv, A.wE, A.wN};
    const double* c[S::NC] = {b, A.diag, A.wU};
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &it.maps, h, c, 1)));
  }
  it.a = typename pf::OpRes<UNI>::Args{g->part, g->st, A.wc, A.diagc, init,
                                       init ? K.r[0] : nullptr, init ? K.rt : nullptr, init ? K.p[0] : nullptr,
                                       init ? K.v[0] : nullptr, init ? K.t : nullptr, g->b32};
  return PF_OK;
}


// ---- batched launches over the members flagged in a map slot -----------------------------------------
template <bool UNI>
pf_status launch_res(pf_batch* B, int op, int init, const int2* map, int grid, cudaStream_t st) {
  using OR = pf::OpResSkip<UNI>;
  const void* items = nullptr;
  PF_TRY((items_for<OR>(B, key_of(init ? "RES1" : "RES0", op, 1, 0),
                        [&](int, pf_grid* g, pf::BatchItem<OR>& it) {
                          return fill_res<UNI>(g, op, init, x_of(g, op), b_of(g, op), it);
                        },
                        &items)));
  return launch_items<OR>(B, items, map, grid, st);
}

template <typename T, bool UNI>
pf_status ca_items(pf_batch* B, int op, int par, int prime, const void** out) {
  using OC = pf::OpCA<T, UNI>;
  constexpr int f64 = sizeof(T) == 8;
  return items_for<OC>(B, key_of(prime ? "CAP" : "CA", op, f64, par),
                       [&](int, pf_grid* g, pf::BatchItem<OC>& it) {
                         T* x;
                         if constexpr (f64) x = x_of(g, op); else x = g->d32;
                         return fill_ca<T, UNI>(g, op, par, prime, x, it);
                       },
                       out);
}

template <typename T, bool UNI>
pf_status launch_prime(pf_batch* B, int op, const int2* map, int grid, cudaStream_t st) {
  const void* items = nullptr;
  PF_TRY((ca_items<T, UNI>(B, op, 0, 1, &items)));
  return launch_items<pf::OpCA<T, UNI>>(B, items, map, grid, st);
}

// TICK_ITERS BiCGSTAB iterations (from parity 1, where every chunk starts) of the members in
// the map slot: one captured graph per operator and precision, replayed while the membership stands; its
// kernel nodes get the tick's grid size (the map's length) when it changes.
template <typename T, bool UNI>
pf_status launch_chunk(pf_batch* B, int op, const int2* map, int grid, cudaStream_t st) {
  using OB = pf::OpB<T, UNI>;
  using OC = pf::OpCA<T, UNI>;
  constexpr int f64 = sizeof(T) == 8;
  const std::string gk = key_of("graph", op, f64, 0);
  auto git = B->graphs.find(gk);
  if (git == B->graphs.end()) {
    const void *ib[2], *ica[2];
    for (int par = 0; par < 2; ++par) {
      PF_TRY((items_for<OB>(B, key_of("B", op, f64, par),
                            [&](int, pf_grid* g, pf::BatchItem<OB>& it) { return fill_b<T, UNI>(g, op, par, it); },
                            &ib[par])));
      PF_TRY((ca_items<T, UNI>(B, op, par, 0, &ica[par])));
    }
    cudaGraph_t graph = nullptr;
    PF_CK(cudaStreamBeginCapture(B->cstream, cudaStreamCaptureModeThreadLocal));
    int cur = 1;
    pf_status ls = PF_OK;
    static_assert(TICK_ITERS % 2 == 0, "chunks start at ping-pong parity 1");
    for (int i = 0; i < TICK_ITERS && ls == PF_OK; ++i) {
      ls = launch_items<OB>(B, ib[cur], map, B->nblocks, B->cstream);
      if (ls == PF_OK) ls = launch_items<OC>(B, ica[cur], map, B->nblocks, B->cstream);
      cur = 1 - cur;
    }
    const cudaError_t ce = cudaStreamEndCapture(B->cstream, &graph);
    if (ls != PF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return ls;
    }
    PF_CK(ce);
    pf_batch::Chunk c;
    c.graph = graph;
    const cudaError_t ie = cudaGraphInstantiate(&c.exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      PF_CK(ie);
    }
    size_t nn = 0;
    PF_CK(cudaGraphGetNodes(graph, nullptr, &nn));
    c.nodes.resize(nn);
    PF_CK(cudaGraphGetNodes(graph, c.nodes.data(), &nn));
    c.grid = B->nblocks;
    git = B->graphs.emplace(gk, c).first;
  }
  pf_batch::Chunk& c = git->second;
  if (grid != c.grid) {
    for (cudaGraphNode_t nd : c.nodes) {
      cudaKernelNodeParams kp;
      PF_CK(cudaGraphKernelNodeGetParams(nd, &kp));
      kp.gridDim = dim3(grid, 1, 1);
      PF_CK(cudaGraphExecKernelNodeSetParams(c.exec, nd, &kp));
    }
    c.grid = grid;
  }
  PF_CK(cudaGraphLaunch(c.exec, st));
  return PF_OK;
}

template <bool UNI>
pf_status launch_kind(pf_batch* B, int op, int kind, const int2* map, int grid, cudaStream_t st) {
  switch (kind) {
    case K_RES0: return launch_res<UNI>(B, op, 0, map, grid, st);
    case K_RES1: return launch_res<UNI>(B, op, 1, map, grid, st);
    case K_PRIME32: return launch_prime<float, UNI>(B, op, map, grid, st);
    case K_PRIME64: return launch_prime<double, UNI>(B, op, map, grid, st);
    case K_CHUNK32: return launch_chunk<float, UNI>(B, op, map, grid, st);
    default: return launch_chunk<double, UNI>(B, op, map, grid, st);
  }
}

// ---- the per-problem state machine ---------------------------------------------------------------
enum Stage { S_NEW = 0, S_FERMI, S_PF2RHS, S_LIN, S_UPDATE, S_FINISH, S_DONE };
enum Sub { L_RES = 0, L_INNER_START, L_INNER, L_START64, L_ITER64 };

// Starts the linear solve of operator op (unknown and right-hand side of x_of / b_of) in this tick.
pf_status lin_start(pf_batch* B, BatchMember& M, int op, int next_stage, double eta) {
  pf_grid* g = M.g;
  M.stage = S_LIN;
  M.after = next_stage;
  M.op = op;
  M.eta = eta;
  M.iters = M.refs = 0;
  M.add_pending = false;
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x_of(g, op), b_of(g, op), ops64(g, op).dinv, g->geom.np, B->stream));
  M.sub = M.o.lin.precision == PF_MIXED ? L_RES : L_START64;
  return PF_OK;
}

// The per-member work of a tick before the batched launches; sets the launch kinds the member takes part in.
pf_status pre(pf_batch* B, BatchMember& M, std::vector<int>& kinds) {
  pf_grid* g = M.g;
  cudaStream_t s = B->stream;
  const long NP = g->geom.np;
  const pf_solve_opts& lo = M.o.lin;
  switch (M.stage) {
    case S_NEW: {
      pf_result& r = *M.res;
      r.status = PF_OK;
      r.outer_iters = r.lin_iters_total = r.lin_iters_first = 0;
      r.delta = 0.0;
      M.U = OuterUpdate{};
      M.dprev = 1.0;
      M.dprev2 = 0.0;
      M.st = PF_OK;
      if (M.o.accel_depth > 0) PF_TRY(ensure_aa(g, M.o.accel_depth));
      if (M.o.predict) PF_TRY(ensure_predict(g));
      PF_TRY(build_operators(g));
      M.fermi_warm = M.o.warm_start && g->ulast_valid;
      if (M.o.warm_start) {  // start from the grid's potential: straight to the first outer iteration
        M.stage = S_FERMI;
        return PF_OK;
      }
      // initial potential (Table 4): PF2 with rho' = Psi = 0
      PF_CK(cudaMemsetAsync(g->phi0, 0, NP * sizeof(double), s));
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_dirichlet(g->phi0, g->lo_hat, g->hi_hat, g->geom, s));
      PF_CK(cudaMemsetAsync(g->psi, 0, NP * sizeof(double), s));
      PF_LAUNCH(g, PF_PROF_OTHER,
                pf::launch_pf2_rhs(g->psi, g->solvent, g->ffix, g->eps_s, g->lo_hat, g->hi_hat, g->geom, g->b2, s));
      PF_TRY(lin_start(B, M, PF_OP_POISSON, S_FERMI, 0.0));
      break;
    }
    case S_FERMI: {
      // Eq. (1) at Phi_0 -> b_PF1, kappa, PF2 right-hand-side part; then PF1 (Eq. 12)
      const int outer = M.res->outer_iters + 1;
      const double eta = M.o.lin_forcing > 0 ? (outer == 1 ? 1e-2 : fmin(1e-2, M.o.lin_forcing * M.dprev)) : 0.0;
      PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
      if (M.o.lin.precision == PF_MIXED)  // double-float on the FP32 pipes, as pf_nonlinear_solve
        PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi_df(g->phi0, g->solvent, g->ffix, g->spd, g->geom, g->b1, g->sig,
                                                        g->c2, g->ulast32, outer > 1 || (M.o.warm_start && g->u32_valid),
                                                        g->err, s));
      else
        PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, g->geom, g->b1, g->sig,
                                                     g->c2, nullptr, nullptr, nullptr, g->ulast,
                                                     outer > 1 || M.fermi_warm, g->err, s));
      PF_TRY(update_pf2(g));
      // starting vectors as pf_nonlinear_solve (pf_nl_opts.predict)
      const bool pred = M.o.predict && outer >= 2;
      M.cpred = (pred && outer >= 3 && M.dprev2 > 0.0 && M.dprev < M.dprev2) ? M.dprev / M.dprev2 : 0.0;
      M.pred_have = M.o.predict == 1 && outer - 1 > 2 ? 2 : outer - 1;
      if (pred) PF_TRY(predict(g, g->psi, g->xp_psi, g->xpp_psi, M.pred_have, M.cpred));
      PF_TRY(lin_start(B, M, PF_OP_PF1, S_PF2RHS, eta));
      break;
    }
    case S_PF2RHS: {
      // PF2 right-hand side from Psi, then PF2 (Eq. 13) from Phi_0
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_pf2_rhs(g->psi, g->solvent, g->c2, g->eps_s, g->lo_hat, g->hi_hat,
                                                     g->geom, g->b2, s));
      if (M.o.predict && M.res->outer_iters >= 1)
        PF_TRY(predict(g, g->phi, g->xp_phi, g->xpp_phi, M.pred_have, M.cpred));  // from the previous PF2 solutions
      else
        PF_CK(cudaMemcpyAsync(g->phi, g->phi0, NP * sizeof(double), cudaMemcpyDeviceToDevice, s));
      PF_TRY(lin_start(B, M, PF_OP_PF2, S_UPDATE, M.eta));
      break;
    }
    case S_FINISH: {
      pf_result& r = *M.res;
      PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
      const bool df_ran = M.o.lin.precision == PF_MIXED && r.outer_iters > 0;
      PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, g->geom, nullptr, nullptr,
                                                   nullptr, g->Cbuf, g->Sbuf, g->Gbuf, g->ulast,
                                                   r.outer_iters > 0 || M.fermi_warm, g->err, s,
                                                   df_ran ? g->ulast32 : nullptr));
      if (df_ran) g->u32_valid = true;
      if (r.phi_V) {  // phi = phi~ + G in the membrane when the charges are decomposed (Eq. 5)
        PF_LAUNCH(g, PF_PROF_OTHER,
                  pf::launch_add_scale(g->phi0, g->charge_mode == 1 ? g->Gdec : nullptr, g->Tv, g->phi, NP, s));
        PF_TRY(unpack_out(g, g->phi, 1, r.phi_V, r.mem));
      }
      if (r.C_M) {
        PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->Cbuf, 1.0 / g->molar, g->Cbuf, NP * g->sp.ns, s));
        PF_TRY(unpack_out(g, g->Cbuf, g->sp.ns, r.C_M, r.mem));
      }
      if (r.S) PF_TRY(unpack_out(g, g->Sbuf, 1, r.S, r.mem));
      if (r.Gamma) PF_TRY(unpack_out(g, g->Gbuf, 1, r.Gamma, r.mem));
      if (r.Psi) PF_TRY(unpack_out(g, g->psi, 1, r.Psi, r.mem));
      PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
      return PF_OK;
    }
    case S_UPDATE:
      return outer_stage1(g, M.U, M.o.accel_depth, M.o.omega);
    default:
      break;
  }
  if (M.stage != S_LIN) return PF_OK;
  const int base = M.op * K_PER_OP;
  switch (M.sub) {
    case L_RES:  // FP64 true residual b - A x -> b32 (mixed precision)
      if (M.add_pending) {
        PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_add_f32(x_of(g, M.op), g->d32, NP, s));  // x += d
        M.add_pending = false;
      }
      PF_TRY(set_state(g, g->st, lo.tol, lo.norm, 0, M.eta, M.refs > 0));
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(b_of(g, M.op), g->geom, g->part, g->st, s));
      kinds.push_back(base + K_RES0);
      break;
    case L_INNER_START: {  // FP32 inner solve A d = r from d = 0 to inner_tol, prime and first chunk
      const Krylov<float> K = kry32(g);
      PF_CK(cudaMemsetAsync(g->d32, 0, NP * sizeof(float), s));
      const int cap = lo.max_iter - M.iters < INNER_CAP ? lo.max_iter - M.iters : INNER_CAP;
      PF_TRY(set_state(g, g->st2, lo.inner_tol, PF_NORM_REL2, cap));
      PF_LAUNCH(g, PF_PROF_INIT, pf::launch_init_zero<float>(g->b32, g->geom, K.r[0], K.rt, K.p[0], K.v[0], K.t,
                                                              g->part, g->st2, s));
      if (M.inner_t2 > 0.0) PF_TRY(raise_tol2(g, g->st2, M.inner_t2, s));  // as pf_nonlinear_solve
      kinds.push_back(base + K_PRIME32);
      kinds.push_back(base + K_CHUNK32);
      M.sub = L_INNER;
      break;
    }
    case L_INNER:
      kinds.push_back(base + K_CHUNK32);
      break;
    case L_START64:  // FP64 BiCGSTAB: r0 = b - A x, prime and first chunk
      PF_TRY(set_state(g, g->st, lo.tol, lo.norm, lo.max_iter, M.eta));
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(b_of(g, M.op), g->geom, g->part, g->st, s));
      kinds.push_back(base + K_RES1);
      kinds.push_back(base + K_PRIME64);
      kinds.push_back(base + K_CHUNK64);
      M.sub = L_ITER64;
      break;
    case L_ITER64:
      kinds.push_back(base + K_CHUNK64);
      break;
  }
  return PF_OK;
}

// Ends the member's linear solve with status ls and moves it on.
void lin_end(BatchMember& M, int ls) {
  if (trace_level() > 0)
    fprintf(stderr, "[pf batch] member %lld op %d linear solve: status %d iters %d refinements %d\n", M.tag, M.op, ls,
            M.iters, M.refs);
  M.res->lin_iters_total += M.iters;
  if (M.op == PF_OP_POISSON) M.res->lin_iters_first = M.iters;
  if (ls != PF_OK) {
    M.st = (pf_status)ls;
    M.stage = S_FINISH;
  } else {
    M.stage = M.after;
  }
}

// The member's transition after the tick's launches landed (states gathered: s64 = st, s32 = st2).
void post(BatchMember& M, const BicgState& s64, const BicgState& s32) {
  const pf_solve_opts& lo = M.o.lin;
  if (M.stage != S_LIN) return;
  switch (M.sub) {
    case L_RES:
      if (s64.done) {
        lin_end(M, PF_OK);
      } else if (!isfinite(s64.rnorm2)) {
        lin_end(M, PF_E_BREAKDOWN);
      } else if (M.refs >= lo.max_refine || M.iters >= lo.max_iter) {
        lin_end(M, PF_E_NOCONV);
      } else {
        M.inner_t2 = final_inner_tol2(lo, s64.rnorm2, s64.tol2);
        M.sub = L_INNER_START;
      }
      break;
    case L_INNER:
      if (s32.done) {
        M.iters += s32.iter;
        ++M.refs;
        if (s32.status == PF_E_BREAKDOWN && s32.iter == 0) {
          lin_end(M, PF_E_BREAKDOWN);
        } else {
          M.add_pending = true;
          M.sub = L_RES;
        }
      }
      break;
    case L_ITER64:
      if (s64.done) {
        M.iters = s64.iter;
        lin_end(M, s64.status);
      }
      break;
    default:
      break;
  }
}

// One tick of the engine over all members.
pf_status tick(pf_batch* B) {
  NvtxRange range("batch tick");
  const auto wall0 = std::chrono::steady_clock::now();
  PF_TRY(build(B));
  cudaStream_t s = B->stream;
  PF_CK(cudaEventRecord(B->tick0, s));
  const int n = (int)B->members.size();
  std::vector<std::vector<int>> kinds(n);
  std::vector<char> use(N_SLOTS, 0);
  // the stage each member was in at the start of the tick (the one whose work this tick runs)
  std::vector<int> was(n);
  for (int i = 0; i < n; ++i) {
    BatchMember& M = B->members[i];
    was[i] = M.stage;
    if (M.stage == S_DONE) continue;
    PF_TRY(pre(B, M, kinds[i]));
    for (int k : kinds[i]) use[k] = 1;
  }
  // block maps of the launch kinds in use: the blocks of the members that take part, nothing else (the
  // previous tick ended with a synchronisation, so the staging area is free)
  const int nb = B->nblocks;
  for (int k = 0; k < SLOT_FULL; ++k) B->mapn[k] = 0;
  for (int i = 0; i < n; ++i)
    for (int k : kinds[i])
      for (int b = 0; b < B->nblk[i]; ++b) B->hmaps[(size_t)k * nb + B->mapn[k]++] = make_int2(i, b);
  for (int k = 0; k < SLOT_FULL; ++k) {
    if (!use[k]) continue;
    const size_t off = (size_t)k * nb * sizeof(int2), bytes = (size_t)B->mapn[k] * sizeof(int2);
    unsigned char* stage = B->harena + ((unsigned char*)B->dmaps - B->darena) + off;
    memcpy(stage, (const unsigned char*)B->hmaps.data() + off, bytes);
    PF_CK(cudaMemcpyAsync((unsigned char*)B->dmaps + off, stage, bytes, cudaMemcpyHostToDevice, s));
  }
  // the batched launches of each operator (residuals, then primes, then the chunk graphs) on the
  // operator's own stream, so that the launches of different operators overlap on the device
  const int order[] = {K_RES0, K_RES1, K_PRIME32, K_PRIME64, K_CHUNK32, K_CHUNK64};
  PF_CK(cudaEventRecord(B->fork, s));
  for (int op = 0; op < N_OPS; ++op) {
    bool any = false;
    for (int kind : order) any = any || use[op * K_PER_OP + kind];
    if (!any) continue;
    cudaStream_t st = B->ops[op];
    PF_CK(cudaStreamWaitEvent(st, B->fork, 0));
    for (int kind : order) {
      const int slot = op * K_PER_OP + kind;
      if (!use[slot]) continue;
      const int2* map = map_of(B, slot);
      const int grid = B->mapn[slot];
      PF_TRY(op == PF_OP_PF1 ? launch_kind<true>(B, op, kind, map, grid, st)
                             : launch_kind<false>(B, op, kind, map, grid, st));
    }
    PF_CK(cudaEventRecord(B->join[op], st));
    PF_CK(cudaStreamWaitEvent(s, B->join[op], 0));
  }
  // every member's states
  pf::k_gather_states<<<(n + 127) / 128, 128, 0, s>>>(B->dst64, B->dst32, n, B->dgather);
  PF_CK(cudaGetLastError());
  PF_CK(cudaMemcpyAsync(B->hgather, B->dgather, 2 * n * sizeof(BicgState), cudaMemcpyDeviceToHost, s));
  PF_CK(cudaEventRecord(B->tick1, s));
  PF_CK(cudaStreamSynchronize(s));
  {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, B->tick0, B->tick1) == cudaSuccess) B->stats.device_ms += ms;
    ++B->stats.ticks;
  }
  // transitions; the outer update's later stages (Anderson inner products, least squares)
  bool dots = false;
  std::vector<char> stop(n, 0);
  for (int i = 0; i < n; ++i) {
    BatchMember& M = B->members[i];
    if (was[i] == S_UPDATE) {
      const double d = outer_delta(M.g, M.o.accel_depth, M.o.omega);
      stop[i] = d <= M.o.tol_outer;
      M.res->delta = d;
      PF_TRY(outer_stage2(M.g, M.U, M.o.accel_depth, stop[i]));
      dots = dots || M.U.dots;
    } else if (was[i] == S_FINISH) {
      if (*M.g->host_err && M.st == PF_OK) M.st = PF_E_GAMMA;
      M.res->status = M.st;
      M.stage = S_DONE;
      M.g->have_phi0 = true;
      M.g->ulast_valid = true;
      prof_resolve(M.g);
    } else {
      post(M, B->hgather[i], B->hgather[n + i]);
    }
  }
  if (dots) PF_CK(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    BatchMember& M = B->members[i];
    if (was[i] != S_UPDATE) continue;
    PF_TRY(outer_stage3(M.g, M.U, M.o.accel_depth, M.o.omega, stop[i]));
    const int outer = ++M.res->outer_iters;
    M.dprev2 = M.dprev;
    M.dprev = M.res->delta;
    if (trace_level() > 0)
      fprintf(stderr, "[pf batch] member %lld outer %d delta %.6e\n", M.tag, outer, M.res->delta);
    if (*M.g->host_err) {
      M.st = PF_E_GAMMA;
      M.stage = S_FINISH;
    } else if (stop[i]) {
      M.stage = S_FINISH;
    } else if (outer >= M.o.max_outer) {
      M.st = PF_E_NOCONV;
      M.stage = S_FINISH;
    } else {
      M.stage = S_FERMI;
    }
  }
  B->stats.wall_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  return PF_OK;
}

// Times the FP32 phase kernels of the batch's Poisson operators (right-hand side: the operator's diagonal
// sums; the FP32 Krylov vectors, the correction and the inner state are scratch until a solve resets them)
// for every tiles-per-block candidate, and keeps the fastest.
pf_status autotune(pf_batch* B) {
  for (pf_grid* g : B->grids) {
    PF_TRY(build_operators(g));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->dsum, g->b32, g->geom.np, B->stream));
  }
  pf_batch_tune t{};
  float best = 1e30f;
  int best_tpb = 4, best_zc = pf::ZC;
  for (int zc : ZC_CANDIDATES)
  for (int c : TPB_CANDIDATES) {
    B->tpb = c;
    B->zc = zc;
    B->built = false;
    PF_TRY(build(B));
    const int2* full = map_of(B, SLOT_FULL);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first pass builds the tables and warms up
      for (pf_grid* g : B->grids) {
        const Krylov<float> K = kry32(g);
        PF_CK(cudaMemsetAsync(g->d32, 0, g->geom.np * sizeof(float), B->stream));
        PF_TRY(set_state(g, g->st2, 1e-30, PF_NORM_REL2, 1000));
        PF_CK(pf::launch_init_zero<float>(g->b32, g->geom, K.r[0], K.rt, K.p[0], K.v[0], K.t, g->part, g->st2,
                                          B->stream));
      }
      using OB = pf::OpB<float, false>;
      using OC = pf::OpCA<float, false>;
      const void *ib[2], *ica[2], *ip;
      for (int par = 0; par < 2; ++par) {
        PF_TRY((items_for<OB>(B, key_of("B", PF_OP_POISSON, 0, par),
                              [&](int, pf_grid* g, pf::BatchItem<OB>& it) {
                                return fill_b<float, false>(g, PF_OP_POISSON, par, it);
                              },
                              &ib[par])));
        PF_TRY((ca_items<float, false>(B, PF_OP_POISSON, par, 0, &ica[par])));
      }
      PF_TRY((ca_items<float, false>(B, PF_OP_POISSON, 0, 1, &ip)));
      PF_CK(cudaEventRecord(B->e0, B->stream));
      PF_TRY(launch_items<OC>(B, ip, full, B->nblocks, B->stream));
      int cur = 1;
      for (int i = 0; i < 4; ++i) {
        PF_TRY(launch_items<OB>(B, ib[cur], full, B->nblocks, B->stream));
        PF_TRY(launch_items<OC>(B, ica[cur], full, B->nblocks, B->stream));
        cur = 1 - cur;
      }
      PF_CK(cudaEventRecord(B->e1, B->stream));
      PF_CK(cudaEventSynchronize(B->e1));
      PF_CK(cudaEventElapsedTime(&ms, B->e0, B->e1));
    }
    if (t.n < PF_BATCH_TUNE_MAX) {
      t.tiles_per_block[t.n] = c;
      t.z_planes[t.n] = zc;
      t.ms[t.n] = ms;
      ++t.n;
    }
    if (ms < best) {
      best = ms;
      best_tpb = c;
      best_zc = zc;
    }
  }
  B->tpb = best_tpb;
  B->zc = best_zc;
  t.chosen = best_tpb;
  t.chosen_z = best_zc;
  B->tune = t;
  B->built = false;
  return PF_OK;
}

pf_status check_nl(const pf_nl_opts& o) {
  PF_TRY(check_opts(o.lin));
  if (o.lin.method != PF_BICGSTAB)
    return fail(PF_E_INVAL, "batches and served requests solve with BiCGSTAB (pf_solve_opts.method = PF_BICGSTAB)");
  if (!(o.omega >= 0 && o.omega < 1) || !(o.tol_outer > 0) || o.max_outer < 1 || o.accel_depth < 0 ||
      o.accel_depth > pf::AA_MAX || !(o.lin_forcing >= 0) || (o.warm_start != 0 && o.warm_start != 1) ||
      o.predict < 0 || o.predict > 2)
    return fail(PF_E_INVAL, "invalid pf_nl_opts");
  return PF_OK;
}

pf_status batch_alloc(cudaStream_t user, int count_hint, pf_batch** out) {
  pf_batch* B = new pf_batch();
  B->user = user;
  B->cap = ARENA_BYTES + (size_t)(count_hint > 0 ? count_hint : 1) * 64 * 1024;
  cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cstream, cudaStreamNonBlocking);
  for (int o = 0; o < N_OPS && e == cudaSuccess; ++o) {
    e = cudaStreamCreateWithFlags(&B->ops[o], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[o], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&B->darena, B->cap);
  if (e == cudaSuccess) e = cudaMallocHost(&B->harena, B->cap);
  if (e == cudaSuccess) e = cudaEventCreate(&B->e0);
  if (e == cudaSuccess) e = cudaEventCreate(&B->e1);
  if (e == cudaSuccess) e = cudaEventCreate(&B->tick0);
  if (e == cudaSuccess) e = cudaEventCreate(&B->tick1);
  if (e != cudaSuccess) {
    pf_batch_destroy(B);
    cudaGetLastError();
    return fail(PF_E_OOM, std::string("batch allocation failed: ") + cudaGetErrorString(e));
  }
  set_attrs<float, false>();
  set_attrs<float, true>();
  set_attrs<double, false>();
  set_attrs<double, true>();
  *out = B;
  return PF_OK;
}

// Gives every grid of the batch the batch's stream while a call runs.
struct StreamSwap {
  pf_batch* B;
  std::vector<cudaStream_t> saved;
  explicit StreamSwap(pf_batch* b) : B(b) {
    for (pf_grid* g : B->grids) {
      saved.push_back(g->stream);
      g->stream = B->stream;
      g->L.stream = B->stream;
    }
  }
  ~StreamSwap() {
    for (size_t i = 0; i < B->grids.size(); ++i) {
      B->grids[i]->stream = saved[i];
      B->grids[i]->L.stream = saved[i];
    }
  }
};

// The batch's stream waits for the work queued on the caller's and the grids' streams.
pf_status enter(pf_batch* B) {
  PF_CK(cudaEventRecord(B->e1, B->user));
  PF_CK(cudaStreamWaitEvent(B->stream, B->e1, 0));
  for (pf_grid* g : B->grids) {
    PF_CK(cudaEventRecord(g->ev1, g->stream));
    PF_CK(cudaStreamWaitEvent(B->stream, g->ev1, 0));
  }
  return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_batch_create(pf_grid* const* grids, int count, void* cuda_stream, pf_batch** out) {
  if (!out) return fail(PF_E_INVAL, "out is NULL");
  *out = nullptr;
  if (!grids || count < 1) return fail(PF_E_INVAL, "need at least one grid");
  for (int i = 0; i < count; ++i) {
    if (!grids[i]) return fail(PF_E_INVAL, "NULL grid in batch");
    for (int j = 0; j < i; ++j)
      if (grids[j] == grids[i]) return fail(PF_E_INVAL, "a grid appears twice in the batch");
  }
  pf_batch* B = nullptr;
  PF_TRY(batch_alloc(static_cast<cudaStream_t>(cuda_stream), count, &B));
  B->grids.assign(grids, grids + count);
  *out = B;
  return PF_OK;
}

pf_status pf_batch_set_tiles_per_block(pf_batch* B, int tiles_per_block) {
  if (!B || tiles_per_block < 0) return fail(PF_E_INVAL, "bad batch or tiles_per_block");
  if (tiles_per_block != B->tpb) invalidate(B);
  B->tpb = tiles_per_block;
  return PF_OK;
}

pf_status pf_batch_set_tiling(pf_batch* B, int tiles_per_block, int z_planes) {
  if (!B || tiles_per_block < 1 || z_planes < 4 || z_planes > 256) return fail(PF_E_INVAL, "bad batch tiling");
  invalidate(B);
  B->tpb = tiles_per_block;
  B->zc = z_planes;
  return PF_OK;
}

pf_status pf_batch_autotune(pf_batch* B, pf_batch_tune* out) {
  if (!B) return fail(PF_E_INVAL, "batch is NULL");
  for (pf_grid* g : B->grids)
    if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first on every grid");
  PF_TRY(enter(B));
  StreamSwap sw(B);
  PF_TRY(autotune(B));
  PF_CK(cudaStreamSynchronize(B->stream));
  if (out) *out = B->tune;
  return PF_OK;
}

pf_status pf_batch_get_tune(pf_batch* B, pf_batch_tune* out) {
  if (!B || !out) return fail(PF_E_INVAL, "batch and out are required");
  *out = B->tune;
  out->chosen = B->tpb;
  out->chosen_z = B->zc;
  return PF_OK;
}

pf_status pf_batch_get_stats(pf_batch* B, pf_batch_stats* out) {
  if (!B || !out) return fail(PF_E_INVAL, "batch and out are required");
  *out = B->stats;
  return PF_OK;
}

pf_status pf_batch_nonlinear_solve(pf_batch* B, const pf_nl_opts* opts, pf_result* results) {
  if (!B || !results) return fail(PF_E_INVAL, "batch and results are required");
  pf_nl_opts o;
  if (opts) o = *opts; else pf_default_nl_opts(&o);
  PF_TRY(check_nl(o));
  const int n = (int)B->grids.size();
  for (int i = 0; i < n; ++i) {
    if (!B->grids[i]->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first on every grid");
    if (B->grids[i]->filter_on) return fail(PF_E_INVAL, "a grid with a filter region cannot be solved in a batch");
    if (o.warm_start && !B->grids[i]->have_phi0)
      return fail(PF_E_INVAL, "warm_start needs a potential on every grid (a previous solve or pf_set_potential)");
    if (results[i].mem != PF_MEM_HOST && results[i].mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "bad result mem");
  }
  PF_TRY(enter(B));
  StreamSwap sw(B);
  cudaStream_t s = B->stream;
  PF_CK(cudaEventRecord(B->e0, s));
  if (B->tpb == 0) PF_TRY(autotune(B));
  B->stats = pf_batch_stats{};
  B->members.assign(n, BatchMember{});
  for (int i = 0; i < n; ++i) {
    B->members[i].g = B->grids[i];
    B->members[i].res = &results[i];
    B->members[i].o = o;
    B->members[i].tag = i;
  }
  // every problem ends within its limits (outer iterations, BiCGSTAB iterations, refinements); the host
  // bound only guards the loop
  const long long limit = 16LL * o.max_outer * (o.lin.max_iter / CHUNK + 4 * o.lin.max_refine + 8) + 64;
  pf_status ts = PF_OK;
  for (long long t = 0;; ++t) {
    bool open = false;
    for (const BatchMember& M : B->members) open = open || M.stage != S_DONE;
    if (!open) break;
    if (t > limit) {
      ts = fail(PF_E_NOCONV, "batched solve exceeded its step bound");
      break;
    }
    ts = tick(B);
    if (ts != PF_OK) break;
  }
  B->members.clear();
  if (ts != PF_OK) return ts;
  PF_CK(cudaEventRecord(B->e1, s));
  PF_CK(cudaEventSynchronize(B->e1));
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, B->e0, B->e1));
  pf_status worst = PF_OK;
  for (int i = 0; i < n; ++i) {
    results[i].time_ms = ms;
    if (results[i].status != PF_OK && worst == PF_OK) worst = (pf_status)results[i].status;
  }
  for (size_t i = 0; i < B->grids.size(); ++i) {
    PF_CK(cudaEventRecord(B->grids[i]->ev1, s));
    PF_CK(cudaStreamWaitEvent(sw.saved[i], B->grids[i]->ev1, 0));
  }
  PF_CK(cudaStreamWaitEvent(B->user, B->e1, 0));
  if (worst != PF_OK) return fail(worst, "a problem of the batch ended with status " + std::to_string((int)worst));
  return PF_OK;
}

pf_status pf_batch_destroy(pf_batch* B) {
  if (!B) return PF_OK;
  drain(B);
  for (auto& kv : B->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  if (B->darena) cudaFree(B->darena);
  if (B->harena) cudaFreeHost(B->harena);
  if (B->dgather) cudaFree(B->dgather);
  if (B->hgather) cudaFreeHost(B->hgather);
  if (B->e0) cudaEventDestroy(B->e0);
  if (B->e1) cudaEventDestroy(B->e1);
  if (B->tick0) cudaEventDestroy(B->tick0);
  if (B->tick1) cudaEventDestroy(B->tick1);
  if (B->fork) cudaEventDestroy(B->fork);
  for (int o = 0; o < N_OPS; ++o) {
    if (B->join[o]) cudaEventDestroy(B->join[o]);
    if (B->ops[o]) cudaStreamDestroy(B->ops[o]);
  }
  if (B->cstream) cudaStreamDestroy(B->cstream);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return PF_OK;
}

}  // extern "C"

// ---- the engine behind the server: members join and leave between ticks -----------------------------
namespace pfi {

pf_status engine_create(int max_members, pf_batch** out) {
  PF_TRY(batch_alloc(nullptr, max_members, out));
  (*out)->tpb = ENGINE_TILES_PER_BLOCK;
  return PF_OK;
}

cudaStream_t engine_stream(pf_batch* B) { return B->stream; }

pf_status engine_add(pf_batch* B, pf_grid* g, pf_result* res, const pf_nl_opts& o, long long tag) {
  if (!g || !res || !g->have_coeffs) return fail(PF_E_INVAL, "engine member needs a grid with coefficients");
  if (g->filter_on) return fail(PF_E_INVAL, "a grid with a filter region cannot join a batch");
  PF_TRY(check_nl(o));
  if (g->stream != B->stream) return fail(PF_E_INVAL, "engine member must use the engine's stream");
  if (o.warm_start && !g->have_phi0) return fail(PF_E_INVAL, "warm_start needs a potential on the grid");
  BatchMember M;
  M.g = g;
  M.res = res;
  M.o = o;
  M.tag = tag;
  B->members.push_back(M);
  B->grids.push_back(g);
  B->built = false;
  return PF_OK;
}

pf_status engine_step(pf_batch* B, std::vector<long long>* finished) {
  PF_TRY(tick(B));
  std::vector<BatchMember> keep;
  std::vector<pf_grid*> kg;
  for (const BatchMember& M : B->members) {
    if (M.stage == S_DONE) {
      finished->push_back(M.tag);
    } else {
      keep.push_back(M);
      kg.push_back(M.g);
    }
  }
  if (keep.size() != B->members.size()) {
    B->members.swap(keep);
    B->grids.swap(kg);
    B->built = false;
  }
  return PF_OK;
}

}  // namespace pfi
