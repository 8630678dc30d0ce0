// pf_batch.cu -- many independent PF problems solved together (pf_batch_*): every BiCGSTAB phase and
// every FP64 residual of all grids of the batch runs as ONE launch of a batched stencil kernel, and the
// chunks of BiCGSTAB iterations between two host checks are replayed as a captured CUDA graph.
//
// The batched kernel gives each grid a contiguous range of blocks (a block map, block -> grid): nblk
// blocks for a grid of ntiles tiles, nblk = ceil(ntiles / tiles_per_block), so a block works for one grid
// only and reduces into that grid's partials and state exactly as the single-grid kernel does.  A grid's
// reduction order therefore depends only on its own size and tiles_per_block: a problem gives bitwise the
// same result alone in a batch or in any mix.  tiles_per_block is picked by timing the FP32 phase kernels
// of the batch's own operators for each candidate (pf_batch_autotune), or set by the caller.  The tensor
// maps and arguments of all grids live in a device table that the blocks read at start.  Grids whose
// solve has finished have their state marked done and their blocks return at once.
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

template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB)
    k_stencil_batch(const BatchItem<Op>* __restrict__ items, const int* __restrict__ block_item,
                    unsigned long long wait_limit) {
  const int i = block_item[blockIdx.x];
  if (i < 0) return;
  const BatchItem<Op>* it = items + i;
  __shared__ typename Op::Args sa;
  __shared__ Geom sg;
  __shared__ int sn[3];
  if (threadIdx.x == 0) {
    sa = it->a;
    sg = it->g;
    sn[0] = it->ntiles;
    sn[1] = (int)blockIdx.x - it->block0;
    sn[2] = it->nblk;
#pragma unroll
    for (int h = 0; h < Op::NH; ++h) tensormap_acquire(&it->maps.h[h]);
#pragma unroll
    for (int c = 0; c < Op::NC; ++c) tensormap_acquire(&it->maps.c[c]);
  }
  __syncthreads();
  stencil_run<Op>(&it->maps, sa, sg, sn[0], sn[1], sn[2], wait_limit);
}

__global__ void k_gather_states(BicgState* const* __restrict__ src, int n, BicgState* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = *src[i];
}

}  // namespace pf

using namespace pfi;
using pf::BicgState;

struct pf_batch {
  std::vector<pf_grid*> grids;
  cudaStream_t user = nullptr;    // the caller's stream
  cudaStream_t stream = nullptr;  // the batch's own stream (graphs are captured on it)
  int tpb = 0;  // tiles per block; 0: tune at the next solve
  pf_batch_tune tune{};
  // launch descriptors: a device arena filled from a pinned staging copy
  unsigned char* darena = nullptr;
  unsigned char* harena = nullptr;
  size_t cap = 0, top = 0;
  std::map<std::string, const void*> items;  // launch kind -> device item table
  std::map<std::string, cudaGraphExec_t> graphs;
  // the grids of the current launch set, in batch order, with their block map
  std::vector<int> set;
  int set_tpb = -1;
  const int* dmap = nullptr;
  int nblocks = 0;
  BicgState** dst_fp64 = nullptr;  // device arrays of the set's state pointers
  BicgState** dst_fp32 = nullptr;
  BicgState* dgather = nullptr;    // gathered states (device) and their pinned host copy
  BicgState* hgather = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

constexpr size_t ARENA_BYTES = 16u << 20;
const int TPB_CANDIDATES[] = {1, 2, 4, 8, 16, 32};

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

void drop_launches(pf_batch* B) {
  cudaStreamSynchronize(B->stream);
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  B->graphs.clear();
  B->items.clear();
  B->top = 0;
  B->set.clear();
  B->set_tpb = -1;
  B->dmap = nullptr;
}

// Copies host bytes into the arena (after the stream has drained, so no queued copy still reads the
// staging area); nullptr when the arena is full.
const void* upload(pf_batch* B, const void* src, size_t bytes) {
  const size_t at = (B->top + 255) / 256 * 256;
  if (at + bytes > B->cap) return nullptr;
  cudaStreamSynchronize(B->stream);
  memcpy(B->harena + at, src, bytes);
  if (cudaMemcpyAsync(B->darena + at, B->harena + at, bytes, cudaMemcpyHostToDevice, B->stream) != cudaSuccess)
    return nullptr;
  B->top = at + bytes;
  return B->darena + at;
}

int blocks_for(int ntiles, int tpb) {
  int b = (ntiles + tpb - 1) / tpb;
  const int cap = pf::max_partial_blocks();
  if (b > cap) b = cap;
  if (b > ntiles) b = ntiles;
  return b < 1 ? 1 : b;
}

// Makes `set` (indices into the batch, in order) the current launch set: block map and state pointers.
pf_status use_set(pf_batch* B, const std::vector<int>& set) {
  if (set == B->set && B->set_tpb == B->tpb && B->dmap) return PF_OK;
  drop_launches(B);
  std::vector<int> map;
  for (size_t j = 0; j < set.size(); ++j) {
    const pf_grid* g = B->grids[set[j]];
    const int nb = blocks_for(g->L.ntiles, B->tpb);
    for (int b = 0; b < nb; ++b) map.push_back((int)j);
  }
  B->dmap = static_cast<const int*>(upload(B, map.data(), map.size() * sizeof(int)));
  std::vector<BicgState*> s64, s32;
  for (int i : set) {
    s64.push_back(B->grids[i]->st);
    s32.push_back(B->grids[i]->st2);
  }
  B->dst_fp64 = (BicgState**)upload(B, s64.data(), s64.size() * sizeof(BicgState*));
  B->dst_fp32 = (BicgState**)upload(B, s32.data(), s32.size() * sizeof(BicgState*));
  if (!B->dmap || !B->dst_fp64 || !B->dst_fp32) return fail(PF_E_OOM, "batch launch table does not fit");
  B->nblocks = (int)map.size();
  B->set = set;
  B->set_tpb = B->tpb;
  return PF_OK;
}

// The item table of one launch kind over the current set, built on first use.
template <class Op, class Fill>
pf_status items_for(pf_batch* B, const std::string& key, Fill fill, const void** out) {
  auto it = B->items.find(key);
  if (it != B->items.end()) {
    *out = it->second;
    return PF_OK;
  }
  std::vector<pf::BatchItem<Op>> v(B->set.size());
  int block0 = 0;
  for (size_t j = 0; j < B->set.size(); ++j) {
    pf_grid* g = B->grids[B->set[j]];
    PF_TRY(fill(g, v[j]));
    v[j].g = g->geom;
    v[j].ntiles = g->L.ntiles;
    v[j].nblk = blocks_for(g->L.ntiles, B->tpb);
    v[j].block0 = block0;
    block0 += v[j].nblk;
  }
  const void* d = upload(B, v.data(), v.size() * sizeof(v[0]));
  if (!d) return fail(PF_E_OOM, "batch launch table does not fit");
  B->items[key] = d;
  *out = d;
  return PF_OK;
}

template <class Op>
pf_status launch_items(pf_batch* B, const void* items) {
  static_assert(pf::scratch_fits<Op>(), "reduction scratch must fit in the stage ring");
  pf::k_stencil_batch<Op><<<B->nblocks, pf::NTHREADS, pf::smem_bytes<Op>(), B->stream>>>(
      static_cast<const pf::BatchItem<Op>*>(items), B->dmap, WAIT_LIMIT);
  PF_CK(cudaGetLastError());
  return PF_OK;
}

template <class Op>
void set_smem_attr() {
  cudaFuncSetAttribute(pf::k_stencil_batch<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf::smem_bytes<Op>());
}

template <typename T, bool UNI>
void set_attrs() {
  set_smem_attr<pf::OpB<T, UNI>>();
  set_smem_attr<pf::OpCA<T, UNI>>();
  if constexpr (sizeof(T) == 8) set_smem_attr<pf::OpResSkip<UNI>>();
}

std::string key_of(const char* kind, int op, int f64, int par, const void* x, const void* b) {
  char buf[128];
  snprintf(buf, sizeof buf, "%s|%d|%d|%d|%p|%p", kind, op, f64, par, x, b);
  return buf;
}

// ---- item fillers (the same arrays, in the same slots, as the single-grid launches)
template <typename T, bool UNI>
pf_status fill_b(pf_grid* g, int op, int cur, pf::BatchItem<pf::OpB<T, UNI>>& it) {
  using SB = pf::SlotsB<UNI>;
  const OpArrays<T> A = opsT<T>(g, op);
  const Krylov<T> K = kryT<T>(g);
  if constexpr (UNI) {
    const T* h[SB::NH] = {K.r[cur], K.v[cur], A.dinv};
    const T* c[SB::NC] = {K.rt};
    PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &it.maps, h, c)));
  } else {
    const T* h[SB::NH] = {K.r[cur], K.v[cur], A.dinv, A.wE, A.wN};
    const T* c[SB::NC] = {K.rt, A.wU};
    PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &it.maps, h, c)));
  }
  it.a = typename pf::OpB<T, UNI>::Args{g->part, sizeof(T) == 8 ? g->st : g->st2, K.t, (T)A.wc};
  return PF_OK;
}

template <typename T, bool UNI>
pf_status fill_ca(pf_grid* g, int op, int cur, int prime, T* x, pf::BatchItem<pf::OpCA<T, UNI>>& it) {
  using SC = pf::SlotsCA<UNI>;
  const OpArrays<T> A = opsT<T>(g, op);
  const Krylov<T> K = kryT<T>(g);
  if constexpr (UNI) {
    const T* h[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv};
    const T* c[SC::NC] = {x, K.rt};
    PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &it.maps, h, c)));
  } else {
    const T* h[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv, A.wE, A.wN};
    const T* c[SC::NC] = {x, K.rt, A.wU};
    PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &it.maps, h, c)));
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
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &it.maps, h, c)));
  } else {
    const double* h[S::NH] = {x, A.dinv, A.wE, A.wN};
    const double* c[S::NC] = {b, A.diag, A.wU};
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &it.maps, h, c)));
  }
  it.a = typename pf::OpRes<UNI>::Args{g->part, g->st, A.wc, A.diagc, init,
                                       init ? K.r[0] : nullptr, init ? K.rt : nullptr, init ? K.p[0] : nullptr,
                                       init ? K.v[0] : nullptr, init ? K.t : nullptr, g->b32};
  return PF_OK;
}

// One unknown of a batched linear solve.
struct Job {
  int inst;          // index in the batch
  double* x;         // unknown (in: start, out: solution)
  const double* b;   // right-hand side
  double eta = 0.0;  // forcing: also stop at eta ||r0||
  int iters = 0, refs = 0;
  int status = PF_OK;
  bool running = true;
};

pf_status gather(pf_batch* B, bool fp32, std::vector<BicgState>& out) {
  const int n = (int)B->set.size();
  pf::k_gather_states<<<(n + 127) / 128, 128, 0, B->stream>>>(fp32 ? B->dst_fp32 : B->dst_fp64, n, B->dgather);
  PF_CK(cudaGetLastError());
  PF_CK(cudaMemcpyAsync(B->hgather, B->dgather, n * sizeof(BicgState), cudaMemcpyDeviceToHost, B->stream));
  PF_CK(cudaStreamSynchronize(B->stream));
  out.assign(B->hgather, B->hgather + n);
  return PF_OK;
}

// BiCGSTAB iterations of the current set (prime, then chunks of [B, C+A] pairs replayed as one graph)
// until every grid's state is done.  x is the FP64 unknown of each job (FP64) or the FP32 correction.
template <typename T, bool UNI>
pf_status batch_iterate(pf_batch* B, int op, const std::vector<Job>& jobs, int max_iter, std::vector<BicgState>& fin) {
  constexpr int f64 = sizeof(T) == 8;
  using OB = pf::OpB<T, UNI>;
  using OC = pf::OpCA<T, UNI>;
  // the unknowns of the set, in set order (FP32: the corrections)
  auto xof = [&](pf_grid* g, size_t j) -> T* {
    if constexpr (f64) return jobs[j].x; else return g->d32;
  };
  const void* x0key = f64 ? (const void*)jobs[0].x : (const void*)B->grids[jobs[0].inst]->d32;
  const void *ib[2], *ica[2], *iprime;
  size_t jj = 0;
  for (int par = 0; par < 2; ++par) {
    PF_TRY((items_for<OB>(B, key_of("B", op, f64, par, x0key, nullptr),
                          [&](pf_grid* g, pf::BatchItem<OB>& it) { return fill_b<T, UNI>(g, op, par, it); },
                          &ib[par])));
    jj = 0;
    PF_TRY((items_for<OC>(B, key_of("CA", op, f64, par, x0key, nullptr),
                          [&](pf_grid* g, pf::BatchItem<OC>& it) { return fill_ca<T, UNI>(g, op, par, 0, xof(g, jj++), it); },
                          &ica[par])));
  }
  jj = 0;
  PF_TRY((items_for<OC>(B, key_of("CAprime", op, f64, 0, x0key, nullptr),
                        [&](pf_grid* g, pf::BatchItem<OC>& it) { return fill_ca<T, UNI>(g, op, 0, 1, xof(g, jj++), it); },
                        &iprime)));
  PF_TRY(launch_items<OC>(B, iprime));
  // the chunk graph: CHUNK iterations starting at parity 1 (CHUNK is even, so every chunk starts there)
  const std::string gk = key_of("graph", op, f64, 0, x0key, nullptr);
  auto git = B->graphs.find(gk);
  cudaGraphExec_t exec = nullptr;
  if (git != B->graphs.end()) {
    exec = git->second;
  } else {
    cudaGraph_t graph = nullptr;
    PF_CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    int cur = 1;
    pf_status ls = PF_OK;
    for (int i = 0; i < CHUNK && ls == PF_OK; ++i) {
      ls = launch_items<OB>(B, ib[cur]);
      if (ls == PF_OK) ls = launch_items<OC>(B, ica[cur]);
      cur = 1 - cur;
    }
    const cudaError_t ce = cudaStreamEndCapture(B->stream, &graph);
    if (ls != PF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return ls;
    }
    PF_CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    PF_CK(ie);
    B->graphs[gk] = exec;
  }
  // every state ends within max_iter iterations (its own limit); the host bound only guards the loop
  for (long chunk = 0; chunk <= max_iter / CHUNK + 2; ++chunk) {
    PF_CK(cudaGraphLaunch(exec, B->stream));
    PF_TRY(gather(B, !f64, fin));
    bool all = true;
    for (size_t j = 0; j < fin.size(); ++j) all = all && fin[j].done;
    if (all) return PF_OK;
  }
  return fail(PF_E_NOCONV, "batched BiCGSTAB did not finish within its iteration limit");
}

// The FP64 residual b - A x of every running job (init: also start BiCGSTAB in the FP64 Krylov vectors).
// Each running job's state must have been reset; the others are marked done and skipped.
template <bool UNI>
pf_status batch_residual(pf_batch* B, int op, std::vector<Job>& jobs, int init) {
  using OR = pf::OpResSkip<UNI>;
  const void* items = nullptr;
  size_t jj = 0;
  PF_TRY((items_for<OR>(B, key_of(init ? "RES1" : "RES0", op, 1, 0, jobs[0].x, jobs[0].b),
                        [&](pf_grid* g, pf::BatchItem<OR>& it) {
                          const Job& J = jobs[jj++];
                          return fill_res<UNI>(g, op, init, J.x, J.b, it);
                        },
                        &items)));
  return launch_items<OR>(B, items);
}

template <bool UNI>
pf_status batch_solve_fp64(pf_batch* B, int op, std::vector<Job>& jobs, const pf_solve_opts& o) {
  for (Job& J : jobs) {
    pf_grid* g = B->grids[J.inst];
    const OpArrays<double> A = ops64(g, op);
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(J.x, J.b, A.dinv, g->geom.np, B->stream));
    PF_TRY(set_state(g, g->st, o.tol, o.norm, o.max_iter, J.eta));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(J.b, g->geom, g->st, B->stream));
  }
  PF_TRY(batch_residual<UNI>(B, op, jobs, 1));
  std::vector<BicgState> fin;
  PF_TRY((batch_iterate<double, UNI>(B, op, jobs, o.max_iter, fin)));
  for (size_t j = 0; j < jobs.size(); ++j) {
    jobs[j].iters = fin[j].iter;
    jobs[j].status = fin[j].status;
  }
  return PF_OK;
}

template <bool UNI>
pf_status batch_solve_mixed(pf_batch* B, int op, std::vector<Job>& jobs, const pf_solve_opts& o) {
  for (Job& J : jobs) {
    pf_grid* g = B->grids[J.inst];
    const OpArrays<double> A = ops64(g, op);
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(J.x, J.b, A.dinv, g->geom.np, B->stream));
    J.running = true;
    J.iters = J.refs = 0;
    J.status = PF_E_NOCONV;
  }
  std::vector<BicgState> st;
  for (;;) {
    // FP64 true residual of the jobs still refining -> b32 (the others are skipped)
    for (Job& J : jobs) {
      pf_grid* g = B->grids[J.inst];
      if (J.running) {
        PF_TRY(set_state(g, g->st, o.tol, o.norm, 0, J.eta, J.refs > 0));
        PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(J.b, g->geom, g->st, B->stream));
      } else {
        PF_CK(pf::launch_mark_done(g->st, B->stream));
      }
    }
    PF_TRY(batch_residual<UNI>(B, op, jobs, 0));
    PF_TRY(gather(B, false, st));
    bool any = false;
    for (size_t j = 0; j < jobs.size(); ++j) {
      Job& J = jobs[j];
      if (!J.running) continue;
      if (st[j].done) {
        J.status = PF_OK;
        J.running = false;
      } else if (!isfinite(st[j].rnorm2)) {
        J.status = PF_E_BREAKDOWN;
        J.running = false;
      } else if (J.refs >= o.max_refine || J.iters >= o.max_iter) {
        J.status = PF_E_NOCONV;
        J.running = false;
      }
      any = any || J.running;
    }
    if (!any) break;
    // FP32 inner solves A d = r of the running jobs from d = 0 to inner_tol (the others skip)
    for (Job& J : jobs) {
      pf_grid* g = B->grids[J.inst];
      if (!J.running) {
        PF_CK(pf::launch_mark_done(g->st2, B->stream));
        continue;
      }
      const Krylov<float> K = kry32(g);
      PF_CK(cudaMemsetAsync(g->d32, 0, g->geom.np * sizeof(float), B->stream));
      const int cap = o.max_iter - J.iters < INNER_CAP ? o.max_iter - J.iters : INNER_CAP;
      PF_TRY(set_state(g, g->st2, o.inner_tol, PF_NORM_REL2, cap));
      PF_LAUNCH(g, PF_PROF_INIT, pf::launch_init_zero<float>(g->b32, g->geom, K.r[0], K.rt, K.p[0], K.v[0], K.t,
                                                              g->part, g->st2, B->stream));
    }
    std::vector<BicgState> fin;
    PF_TRY((batch_iterate<float, UNI>(B, op, jobs, INNER_CAP, fin)));
    for (size_t j = 0; j < jobs.size(); ++j) {
      Job& J = jobs[j];
      if (!J.running) continue;
      pf_grid* g = B->grids[J.inst];
      J.iters += fin[j].iter;
      ++J.refs;
      if (fin[j].status == PF_E_BREAKDOWN && fin[j].iter == 0) {
        J.status = PF_E_BREAKDOWN;
        J.running = false;
        continue;
      }
      PF_LAUNCH(g, PF_PROF_RESIDUAL, pf::launch_add_f32(J.x, g->d32, g->geom.np, B->stream));  // x += d
    }
  }
  return PF_OK;
}

// A batched linear solve of the given jobs (one operator for all).
pf_status batch_solve(pf_batch* B, int op, std::vector<Job>& jobs, const pf_solve_opts& o) {
  if (jobs.empty()) return PF_OK;
  std::vector<int> set;
  for (const Job& J : jobs) set.push_back(J.inst);
  PF_TRY(use_set(B, set));
  const bool uni = op == PF_OP_PF1;
  if (o.precision == PF_MIXED)
    return uni ? batch_solve_mixed<true>(B, op, jobs, o) : batch_solve_mixed<false>(B, op, jobs, o);
  return uni ? batch_solve_fp64<true>(B, op, jobs, o) : batch_solve_fp64<false>(B, op, jobs, o);
}

// Times the FP32 phase kernels of the batch's Poisson operators (right-hand side: the operator's diagonal
// sums; the FP32 Krylov vectors, the correction and the inner state are scratch until a solve resets them)
// for every tiles-per-block candidate, and keeps the fastest.
pf_status autotune(pf_batch* B) {
  const int n = (int)B->grids.size();
  std::vector<int> all(n);
  for (int i = 0; i < n; ++i) all[i] = i;
  for (pf_grid* g : B->grids) {
    PF_TRY(build_operators(g));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->dsum, g->b32, g->geom.np, B->stream));
  }
  pf_batch_tune t{};
  float best = 1e30f;
  int best_tpb = 4;
  for (int c : TPB_CANDIDATES) {
    B->tpb = c;
    PF_TRY(use_set(B, all));
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
        PF_TRY((items_for<OB>(B, key_of("B", PF_OP_POISSON, 0, par, nullptr, nullptr),
                              [&](pf_grid* g, pf::BatchItem<OB>& it) { return fill_b<float, false>(g, PF_OP_POISSON, par, it); },
                              &ib[par])));
        PF_TRY((items_for<OC>(B, key_of("CA", PF_OP_POISSON, 0, par, nullptr, nullptr),
                              [&](pf_grid* g, pf::BatchItem<OC>& it) {
                                return fill_ca<float, false>(g, PF_OP_POISSON, par, 0, g->d32, it);
                              },
                              &ica[par])));
      }
      PF_TRY((items_for<OC>(B, key_of("CAprime", PF_OP_POISSON, 0, 0, nullptr, nullptr),
                            [&](pf_grid* g, pf::BatchItem<OC>& it) {
                              return fill_ca<float, false>(g, PF_OP_POISSON, 0, 1, g->d32, it);
                            },
                            &ip)));
      PF_CK(cudaEventRecord(B->e0, B->stream));
      PF_TRY(launch_items<OC>(B, ip));
      int cur = 1;
      for (int i = 0; i < 4; ++i) {
        PF_TRY(launch_items<OB>(B, ib[cur]));
        PF_TRY(launch_items<OC>(B, ica[cur]));
        cur = 1 - cur;
      }
      PF_CK(cudaEventRecord(B->e1, B->stream));
      PF_CK(cudaEventSynchronize(B->e1));
      PF_CK(cudaEventElapsedTime(&ms, B->e0, B->e1));
    }
    if (t.n < PF_BATCH_TUNE_MAX) {
      t.tiles_per_block[t.n] = c;
      t.ms[t.n] = ms;
      ++t.n;
    }
    if (ms < best) {
      best = ms;
      best_tpb = c;
    }
  }
  B->tpb = best_tpb;
  t.chosen = best_tpb;
  B->tune = t;
  drop_launches(B);
  return PF_OK;
}

// Runs f on every grid of the batch with the batch's stream as the grid's stream.
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
  pf_batch* B = new pf_batch();
  B->grids.assign(grids, grids + count);
  B->user = static_cast<cudaStream_t>(cuda_stream);
  B->cap = ARENA_BYTES + (size_t)count * 64 * 1024;
  cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&B->darena, B->cap);
  if (e == cudaSuccess) e = cudaMallocHost(&B->harena, B->cap);
  if (e == cudaSuccess) e = cudaMalloc(&B->dgather, count * sizeof(BicgState));
  if (e == cudaSuccess) e = cudaMallocHost(&B->hgather, count * sizeof(BicgState));
  if (e == cudaSuccess) e = cudaEventCreate(&B->e0);
  if (e == cudaSuccess) e = cudaEventCreate(&B->e1);
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

pf_status pf_batch_set_tiles_per_block(pf_batch* B, int tiles_per_block) {
  if (!B || tiles_per_block < 0) return fail(PF_E_INVAL, "bad batch or tiles_per_block");
  if (tiles_per_block != B->tpb) drop_launches(B);
  B->tpb = tiles_per_block;
  return PF_OK;
}

pf_status pf_batch_autotune(pf_batch* B, pf_batch_tune* out) {
  if (!B) return fail(PF_E_INVAL, "batch is NULL");
  for (pf_grid* g : B->grids)
    if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first on every grid");
  PF_CK(cudaEventRecord(B->e1, B->user));
  PF_CK(cudaStreamWaitEvent(B->stream, B->e1, 0));
  for (pf_grid* g : B->grids) {
    PF_CK(cudaEventRecord(g->ev1, g->stream));
    PF_CK(cudaStreamWaitEvent(B->stream, g->ev1, 0));
  }
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
  return PF_OK;
}

pf_status pf_batch_nonlinear_solve(pf_batch* B, const pf_nl_opts* opts, pf_result* results) {
  if (!B || !results) return fail(PF_E_INVAL, "batch and results are required");
  pf_nl_opts o;
  if (opts) o = *opts; else pf_default_nl_opts(&o);
  PF_TRY(check_opts(o.lin));
  if (!(o.omega >= 0 && o.omega < 1) || !(o.tol_outer > 0) || o.max_outer < 1 || o.accel_depth < 0 ||
      o.accel_depth > pf::AA_MAX || !(o.lin_forcing >= 0))
    return fail(PF_E_INVAL, "invalid pf_nl_opts");
  const int n = (int)B->grids.size();
  const int m = o.accel_depth;
  for (int i = 0; i < n; ++i) {
    if (!B->grids[i]->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first on every grid");
    if (results[i].mem != PF_MEM_HOST && results[i].mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "bad result mem");
  }
  // the batch's stream waits for what is queued on the caller's and the grids' streams, and they wait for
  // the batch at the end
  PF_CK(cudaEventRecord(B->e1, B->user));
  PF_CK(cudaStreamWaitEvent(B->stream, B->e1, 0));
  for (pf_grid* g : B->grids) {
    PF_CK(cudaEventRecord(g->ev1, g->stream));
    PF_CK(cudaStreamWaitEvent(B->stream, g->ev1, 0));
  }
  StreamSwap sw(B);
  cudaStream_t s = B->stream;
  PF_CK(cudaEventRecord(B->e0, s));
  if (B->tpb == 0) PF_TRY(autotune(B));
  std::vector<OuterUpdate> U(n);
  std::vector<double> dprev(n, 1.0);
  std::vector<pf_status> stat(n, PF_OK);
  std::vector<bool> live(n, true);
  for (int i = 0; i < n; ++i) {
    pf_grid* g = B->grids[i];
    pf_result& r = results[i];
    r.status = PF_OK;
    r.outer_iters = r.lin_iters_total = r.lin_iters_first = 0;
    r.delta = 0.0;
    if (m > 0) PF_TRY(ensure_aa(g, m));
    const long NP = g->geom.np;
    PF_TRY(build_operators(g));
    PF_CK(cudaMemsetAsync(g->phi0, 0, NP * sizeof(double), s));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_dirichlet(g->phi0, g->lo_hat, g->hi_hat, g->geom, s));
    PF_CK(cudaMemsetAsync(g->psi, 0, NP * sizeof(double), s));
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_pf2_rhs(g->psi, g->solvent, g->ffix, g->eps_s, g->lo_hat, g->hi_hat, g->geom, g->b2, s));
  }
  // initial potential (Table 4): PF2 with rho' = Psi = 0, all grids in one batched solve
  {
    std::vector<Job> jobs;
    for (int i = 0; i < n; ++i) {
      Job J;
      J.inst = i;
      J.x = B->grids[i]->phi0;
      J.b = B->grids[i]->b2;
      jobs.push_back(J);
    }
    PF_TRY(batch_solve(B, PF_OP_POISSON, jobs, o.lin));
    for (const Job& J : jobs) {
      results[J.inst].lin_iters_first = J.iters;
      results[J.inst].lin_iters_total += J.iters;
      if (J.status != PF_OK) {
        stat[J.inst] = (pf_status)J.status;
        live[J.inst] = false;
      }
    }
  }
  for (int outer = 1; outer <= o.max_outer; ++outer) {
    std::vector<int> act;
    for (int i = 0; i < n; ++i)
      if (live[i]) act.push_back(i);
    if (act.empty()) break;
    std::vector<double> eta(n, 0.0);
    for (int i : act) {
      pf_grid* g = B->grids[i];
      if (o.lin_forcing > 0) eta[i] = outer == 1 ? 1e-2 : fmin(1e-2, o.lin_forcing * dprev[i]);
      // Eq. (1) at Phi_0 -> b_PF1, kappa, PF2 right-hand-side part
      PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
      PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, g->geom, g->b1, g->sig,
                                                   g->c2, nullptr, nullptr, nullptr, g->ulast, outer > 1, g->err, s));
      PF_TRY(update_pf2(g));
    }
    // PF1 (Eq. 12) on every live grid
    std::vector<Job> jobs;
    for (int i : act) {
      Job J;
      J.inst = i;
      J.x = B->grids[i]->psi;
      J.b = B->grids[i]->b1;
      J.eta = eta[i];
      jobs.push_back(J);
    }
    PF_TRY(batch_solve(B, PF_OP_PF1, jobs, o.lin));
    std::vector<Job> jobs2;
    for (const Job& J : jobs) {
      results[J.inst].lin_iters_total += J.iters;
      if (J.status != PF_OK) {
        stat[J.inst] = (pf_status)J.status;
        live[J.inst] = false;
        continue;
      }
      pf_grid* g = B->grids[J.inst];
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_pf2_rhs(g->psi, g->solvent, g->c2, g->eps_s, g->lo_hat, g->hi_hat,
                                                     g->geom, g->b2, s));
      PF_CK(cudaMemcpyAsync(g->phi, g->phi0, g->geom.np * sizeof(double), cudaMemcpyDeviceToDevice, s));
      Job K;
      K.inst = J.inst;
      K.x = g->phi;
      K.b = g->b2;
      K.eta = J.eta;
      jobs2.push_back(K);
    }
    // PF2 (Eq. 13)
    PF_TRY(batch_solve(B, PF_OP_PF2, jobs2, o.lin));
    std::vector<int> upd;
    for (const Job& J : jobs2) {
      results[J.inst].lin_iters_total += J.iters;
      if (J.status != PF_OK) {
        stat[J.inst] = (pf_status)J.status;
        live[J.inst] = false;
        continue;
      }
      upd.push_back(J.inst);
    }
    // the outer update of every grid, stage by stage between two synchronisations
    for (int i : upd) PF_TRY(outer_stage1(B->grids[i], U[i], m, o.omega));
    PF_CK(cudaStreamSynchronize(s));
    std::vector<char> stop(n, 0);
    for (int i : upd) {
      const double d = outer_delta(B->grids[i], m, o.omega);
      stop[i] = d <= o.tol_outer;
      results[i].delta = d;
      PF_TRY(outer_stage2(B->grids[i], U[i], m, stop[i]));
    }
    if (m > 0) PF_CK(cudaStreamSynchronize(s));
    for (int i : upd) {
      pf_grid* g = B->grids[i];
      PF_TRY(outer_stage3(g, U[i], m, o.omega, stop[i]));
      results[i].outer_iters = outer;
      dprev[i] = results[i].delta;
      if (*g->host_err) {
        stat[i] = PF_E_GAMMA;
        live[i] = false;
      } else if (stop[i]) {
        live[i] = false;
      } else if (outer == o.max_outer) {
        stat[i] = PF_E_NOCONV;
        live[i] = false;
      }
    }
  }
  // outputs at the final potentials
  for (int i = 0; i < n; ++i) {
    pf_grid* g = B->grids[i];
    pf_result& r = results[i];
    const long NP = g->geom.np;
    PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, g->geom, nullptr, nullptr,
                                                 nullptr, g->Cbuf, g->Sbuf, g->Gbuf, g->ulast, r.outer_iters > 0,
                                                 g->err, s));
    if (r.phi_V) {
      PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->phi0, g->Tv, g->phi, NP, s));
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
  }
  PF_CK(cudaEventRecord(B->e1, s));
  PF_CK(cudaEventSynchronize(B->e1));
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, B->e0, B->e1));
  pf_status worst = PF_OK;
  for (int i = 0; i < n; ++i) {
    pf_grid* g = B->grids[i];
    if (*g->host_err && stat[i] == PF_OK) stat[i] = PF_E_GAMMA;
    results[i].status = stat[i];
    results[i].time_ms = ms;
    prof_resolve(g);
    if (stat[i] != PF_OK && worst == PF_OK) worst = stat[i];
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
  if (B->stream || B->darena) cudaStreamSynchronize(B->stream);
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  if (B->darena) cudaFree(B->darena);
  if (B->harena) cudaFreeHost(B->harena);
  if (B->dgather) cudaFree(B->dgather);
  if (B->hgather) cudaFreeHost(B->hgather);
  if (B->e0) cudaEventDestroy(B->e0);
  if (B->e1) cudaEventDestroy(B->e1);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return PF_OK;
}

}  // extern "C"
