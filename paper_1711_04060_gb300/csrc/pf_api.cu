// pf_api.cu -- the C ABI of include/pf_gb300.h: grid state, coefficient setup, and the host
// control of the device solvers (Table 3 linear solver, Table 4 nonlinear solver, FP64 iterative
// refinement around FP32 BiCGSTAB).  Every arithmetic step runs in the kernels of pf_kernels.cu;
// this file allocates, encodes the TMA descriptors, launches, and reads back the few scalars that
// steer the iteration.  Device arrays use the padded layout of pf::Geom; caller arrays are compact
// and are packed / unpacked at this boundary.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pf_gb300.h"
#include "pf_cg.cuh"
#include "pf_decomp.cuh"
#include "pf_filter.cuh"
#include "pf_grid.cuh"

using pf::BicgState;

using namespace pfi;

namespace pfi {

thread_local std::string g_err;

pf_status fail(pf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

pf_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return PF_E_CUDA;
}

}  // namespace pfi

namespace {

// Table 1 constants
constexpr double KB = 1.38e-23;        // J/K
constexpr double QE = 1.602e-19;       // C
constexpr double EPS0 = 8.85e-12;      // F/m (8.85e-14 F/cm)
constexpr double NAVO = 6.02214076e23; // 1/mol (SI value; the paper does not print it)

}  // namespace

namespace pfi {

// Small pinned host blocks (for the scalars the host reads back) come from a process-wide free list and are
// never returned to the driver, so no grid's teardown waits on the device.
constexpr size_t PINNED_BLOCK = 4096;
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;

void* pinned_get() {
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  if (g_pinned_free.empty()) {
    unsigned char* slab = nullptr;
    if (cudaMallocHost(&slab, 64 * PINNED_BLOCK) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = 63; i >= 0; --i) g_pinned_free.push_back(slab + i * PINNED_BLOCK);
  }
  void* b = g_pinned_free.back();
  g_pinned_free.pop_back();
  memset(b, 0, PINNED_BLOCK);
  return b;
}

void pinned_put(void* b) {
  if (!b) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.push_back(b);
}

void free_all(pf_grid* g) {
  if (g->dch) cudaFreeAsync(g->dch, g->stream);
  g->dch = nullptr;
  for (cudaEvent_t e : g->pool) cudaEventDestroy(e);
  g->pool.clear();
  for (void* q : g->allocs) cudaFreeAsync(q, g->stream);
  g->allocs.clear();
  pinned_put(g->hostblk);
  g->hostblk = nullptr;
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  g->host_st = nullptr;
  g->host_err = nullptr;
  g->host_delta = nullptr;
  g->aa_host = nullptr;
}

// All arrays of a grid are carved from one allocation (each start 256-byte aligned, as TMA needs 16).
pf_status allocate(pf_grid* g) {
  const long NP = g->geom.np;
  double** d64[] = {&g->eps, &g->wE, &g->wN, &g->wU, &g->dsum, &g->ffix, &g->diagP, &g->dinvP, &g->diag2,
                    &g->dinv2, &g->sig, &g->dinv1, &g->r64[0], &g->r64[1], &g->p64[0], &g->p64[1], &g->v64[0],
                    &g->v64[1], &g->rt64, &g->t64, &g->xb, &g->bb, &g->stage, &g->phi0, &g->phi, &g->psi, &g->b1,
                    &g->c2, &g->b2, &g->Sbuf, &g->Gbuf, &g->ulast};
  float** d32[] = {&g->wE32, &g->wN32, &g->wU32, &g->gh32, &g->dinvP32, &g->dinv2_32, &g->dinv1_32, &g->r32[0], &g->r32[1],
                   &g->p32[0], &g->p32[1], &g->v32[0], &g->v32[1], &g->rt32, &g->t32, &g->d32, &g->b32,
                   &g->ulast32};
  std::vector<std::pair<void**, size_t>> parts;
  for (double** p : d64) parts.push_back({reinterpret_cast<void**>(p), NP * sizeof(double)});
  parts.push_back({reinterpret_cast<void**>(&g->Cbuf), (size_t)NP * pf::MAXSP * sizeof(double)});
  for (float** p : d32) parts.push_back({reinterpret_cast<void**>(p), NP * sizeof(float)});
  parts.push_back({reinterpret_cast<void**>(&g->solvent), (size_t)NP});
  parts.push_back({reinterpret_cast<void**>(&g->part), (size_t)pf::max_partial_blocks() * pf::NPART * sizeof(double)});
  parts.push_back({reinterpret_cast<void**>(&g->st), sizeof(BicgState)});
  parts.push_back({reinterpret_cast<void**>(&g->st2), sizeof(BicgState)});
  parts.push_back({reinterpret_cast<void**>(&g->err), sizeof(int)});
  parts.push_back({reinterpret_cast<void**>(&g->delta), sizeof(double)});
  parts.push_back({reinterpret_cast<void**>(&g->ticket), sizeof(unsigned int)});
  size_t total = 0;
  for (auto& q : parts) total += (q.second + 255) / 256 * 256;
  unsigned char* base = nullptr;
  PF_TRY(dalloc(g, &base, total));
  size_t off = 0;
  for (auto& q : parts) {
    *q.first = base + off;
    off += (q.second + 255) / 256 * 256;
  }
  g->hostblk = pinned_get();
  if (!g->hostblk) return fail(PF_E_OOM, "pinned host allocation failed");
  static_assert(sizeof(BicgState) <= 512, "the pinned block layout holds the state in 512 bytes");
  unsigned char* hb = static_cast<unsigned char*>(g->hostblk);
  g->host_st = reinterpret_cast<BicgState*>(hb);
  g->host_err = reinterpret_cast<int*>(hb + 512);
  g->host_delta = reinterpret_cast<double*>(hb + 1024);
  g->aa_host = reinterpret_cast<double*>(hb + 1536);
  // every array starts at zero: the pad columns and the Krylov vectors on the Dirichlet planes, which no
  // kernel writes, stay zero
  PF_CK(cudaMemsetAsync(base, 0, total, g->stream));
  PF_CK(cudaEventCreate(&g->ev0));
  PF_CK(cudaEventCreate(&g->ev1));
  g->pool.resize(4 * PROF_SLOTS, nullptr);
  g->pkind.resize(2 * PROF_SLOTS, 0);
  for (auto& e : g->pool) PF_CK(cudaEventCreate(&e));
  return PF_OK;
}

// PF_TRACE=1 prints one line per linear solve and outer iteration to stderr, PF_TRACE=2 also one
// line per chunk of BiCGSTAB iterations.
int trace_level() {
  static int lvl = -1;
  if (lvl < 0) {
    const char* e = getenv("PF_TRACE");
    lvl = e ? atoi(e) : 0;
  }
  return lvl;
}

// ---- profiling ---------------------------------------------------------------------------
// read back the first n pairs of half h
static void prof_resolve_half(pf_grid* g, int h, int n) {
  if (n <= 0) return;
  const int b = h * PROF_SLOTS;
  if (cudaEventSynchronize(g->pool[2 * (b + n - 1) + 1]) == cudaSuccess) {
    for (int i = b; i < b + n; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g->pool[2 * i], g->pool[2 * i + 1]) == cudaSuccess) {
        g->pms[g->pkind[i]] += ms;
        g->pcount[g->pkind[i]] += 1;
      }
    }
  }
  cudaGetLastError();
}

void prof_resolve(pf_grid* g) {
  prof_resolve_half(g, g->half ^ 1, g->nold);
  prof_resolve_half(g, g->half, g->np);
  g->nold = 0;
  g->np = 0;
}

int prof_begin(pf_grid* g, int n_launches) {
  g->launches += n_launches;
  if (!g->prof_on) return -1;
  if (g->np == PROF_SLOTS) {  // the current half is full: read back the other one and reuse it
    prof_resolve_half(g, g->half ^ 1, g->nold);
    g->half ^= 1;
    g->nold = PROF_SLOTS;
    g->np = 0;
  }
  cudaEventRecord(g->pool[2 * (g->half * PROF_SLOTS + g->np)], g->stream);
  return g->np;
}

void prof_end(pf_grid* g, int slot, int kind) {
  if (slot < 0) return;
  const int i = g->half * PROF_SLOTS + slot;
  cudaEventRecord(g->pool[2 * i + 1], g->stream);
  g->pkind[i] = kind;
  g->np = slot + 1;
}



// ---- operators -------------------------------------------------------------------------

double pf1_face(const pf_grid* g) { return g->eps_s * g->lc * g->lc / (g->h * g->h); }

OpArrays<double> ops64(const pf_grid* g, int op) {
  if (op == PF_OP_PF1) {
    const double wc = pf1_face(g);
    return {g->dinv1, nullptr, nullptr, nullptr, nullptr, wc, 6.0 * wc + g->eps_s, nullptr};
  }
  return {op == PF_OP_PF2 ? g->dinv2 : g->dinvP, op == PF_OP_PF2 ? g->diag2 : g->diagP, g->wE, g->wN, g->wU, 0.0, 0.0,
          nullptr};
}

OpArrays<float> ops32(const pf_grid* g, int op) {
  if (op == PF_OP_PF1) {
    const double wc = pf1_face(g);
    return {g->dinv1_32, nullptr, nullptr, nullptr, nullptr, wc, 6.0 * wc + g->eps_s, nullptr};
  }
  return {op == PF_OP_PF2 ? g->dinv2_32 : g->dinvP32, nullptr, g->wE32, g->wN32, g->wU32, 0.0, 0.0, g->gh32};
}

pf_status set_state(pf_grid* g, BicgState* dst, double tol, int norm, int max_iter, double tol_r0,
                    int keep_r0) {
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_state(dst, tol, norm, max_iter, tol_r0, keep_r0, g->stream));
  return PF_OK;
}

pf_status read_state(pf_grid* g, const BicgState* src, BicgState* out) {
  PF_CK(cudaMemcpyAsync(g->host_st, src, sizeof(BicgState), cudaMemcpyDeviceToHost, g->stream));
  PF_CK(cudaStreamSynchronize(g->stream));
  *out = *g->host_st;
  return PF_OK;
}


Krylov<double> kry64(pf_grid* g) { return {{g->r64[0], g->r64[1]}, {g->p64[0], g->p64[1]}, {g->v64[0], g->v64[1]}, g->rt64, g->t64}; }
Krylov<float> kry32(pf_grid* g) { return {{g->r32[0], g->r32[1]}, {g->p32[0], g->p32[1]}, {g->v32[0], g->v32[1]}, g->rt32, g->t32}; }

// FP64 residual r = b - A x over the operator: init = 1 starts BiCGSTAB (r, r~, p = v = t = 0 in K),
// init = 0 writes (float) r to b32 for iterative refinement.  The state must have been reset.
template <bool UNI>
pf_status residual(pf_grid* g, const OpArrays<double>& A, const double* x, const double* b, int init,
                   const Krylov<double>* K, BicgState* st, const pf::ResidualExtras& ex = pf::ResidualExtras()) {
  using S = pf::SlotsRes<UNI>;
  pf::Maps<S::NH, S::NC> m;
  if constexpr (UNI) {
    const double* h[S::NH] = {x, A.dinv};
    const double* c[S::NC] = {b};
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &m, h,
                                            c)));
  } else {
    const double* h[S::NH] = {x, A.dinv, A.wE, A.wN};
    const double* c[S::NC] = {b, A.diag, A.wU};
    PF_TRY((fill_maps<S::NH, S::NC, double>(g, &m, h,
                                            c)));
  }
  if (ex.need_bb) PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(b, g->geom, g->part, st, g->stream));
  const int slot = prof_begin(g, 1);
  PF_CK((pf::launch_residual<UNI>(m, g->geom, A.wc, A.diagc, init, K ? K->r[0] : nullptr, K ? K->rt : nullptr,
                                  K ? K->p[0] : nullptr, K ? K->v[0] : nullptr, K ? K->t : nullptr, g->b32, g->part,
                                  st, g->L, ex)));
  prof_end(g, slot, init ? PF_PROF_INIT : PF_PROF_RESIDUAL);
  return PF_OK;
}

// BiCGSTAB iterations (prime, then [B, C+A] pairs in chunks) after the start kernel has written r0 = r[0],
// r~, p[0] = v[0] = t = 0 and started the state.  Returns the final device state in *out.
template <typename T, bool UNI>
pf_status iterate(pf_grid* g, const OpArrays<T>& A, T* x, const Krylov<T>& K, BicgState* st, BicgState* out) {
  using SB = pf::SlotsB<T, UNI>;
  using SC = pf::SlotsCA<T, UNI>;
  const bool f64 = sizeof(T) == 8;
  const int kb = UNI ? (f64 ? PF_PROF_B_FP64_PF1 : PF_PROF_B_FP32_PF1) : (f64 ? PF_PROF_B_FP64 : PF_PROF_B_FP32);
  const int kca = UNI ? (f64 ? PF_PROF_CA_FP64_PF1 : PF_PROF_CA_FP32_PF1) : (f64 ? PF_PROF_CA_FP64 : PF_PROF_CA_FP32);
  // descriptors for the two parities of the ping-pong vectors (r, p, v of iteration parity `cur`)
  pf::Maps<SB::NH, SB::NC> mb[2];
  pf::Maps<SC::NH, SC::NC> mca[2];
  for (int cur = 0; cur < 2; ++cur) {
    if constexpr (UNI) {
      const T* hb[SB::NH] = {K.r[cur], K.v[cur], A.dinv};
      const T* cb[SB::NC] = {K.rt};
      PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &mb[cur], hb,
                                           cb)));
      const T* hc[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv};
      const T* cc[SC::NC] = {x, K.rt};
      PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &mca[cur], hc,
                                           cc)));
    } else if constexpr (pf::ca_face_from_gh<T>()) {
      const T* hb[SB::NH] = {K.r[cur], K.v[cur], A.dinv, A.wE, A.wN};
      const T* cb[SB::NC] = {K.rt, A.wU};
      PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &mb[cur], hb, cb)));
      const T* hc[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv, A.gh};
      const T* cc[SC::NC] = {x, K.rt};
      PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &mca[cur], hc, cc)));
    } else {
      const T* hb[SB::NH] = {K.r[cur], K.v[cur], A.dinv, A.wE, A.wN};
      const T* cb[SB::NC] = {K.rt, A.wU};
      PF_TRY((fill_maps<SB::NH, SB::NC, T>(g, &mb[cur], hb,
                                           cb)));
      const T* hc[SC::NH] = {K.r[cur], K.v[cur], K.t, K.p[cur], A.dinv, A.wE, A.wN};
      const T* cc[SC::NC] = {x, K.rt, A.wU};
      PF_TRY((fill_maps<SC::NH, SC::NC, T>(g, &mca[cur], hc,
                                           cc)));
    }
  }
  const T wc = (T)A.wc;
  PF_LAUNCH(g, kca, (pf::launch_phase_ca<T, UNI>(mca[0], g->geom, wc, x, K.r[1], K.p[1], K.v[1], g->part, st, 1, g->L)));
  int cur = 1;
  for (;;) {
    for (int i = 0; i < CHUNK; ++i) {
      PF_LAUNCH(g, kb, (pf::launch_phase_b<T, UNI>(mb[cur], g->geom, wc, K.t, g->part, st, g->L)));
      PF_LAUNCH(g, kca, (pf::launch_phase_ca<T, UNI>(mca[cur], g->geom, wc, x, K.r[1 - cur], K.p[1 - cur],
                                                     K.v[1 - cur], g->part, st, 0, g->L)));
      cur = 1 - cur;
    }
    BicgState s;
    PF_TRY(read_state(g, st, &s));
    if (trace_level() > 1)
      fprintf(stderr, "[pf] %s it %d rel %.3e rho %.3e alpha %.3e omega %.3e done %d status %d\n",
              f64 ? "fp64" : "fp32", s.iter, sqrt(s.rnorm2 / (s.bnorm2 > 0 ? s.bnorm2 : 1.0)), s.rho, s.alpha,
              s.omega, s.done, s.status);
    if (s.done) {
      *out = s;
      return PF_OK;
    }
  }
}

// Conjugate gradients (one pass per iteration, OpCG) after the start kernel has written r0 = r[0] and zeroed
// w = v[0], s = p[0] and p = t and started the state: the prime pass, then chunks of CHUNK passes between reads of
// the device state.  The Krylov vectors of BiCGSTAB serve: r <- r[], w <- v[], s <- p[], p <- t.
template <typename T, bool UNI>
pf_status iterate_cg(pf_grid* g, const OpArrays<T>& A, T* x, const Krylov<T>& K, BicgState* st, BicgState* out) {
  using S = pf::SlotsCG<T, UNI>;
  const bool f64 = sizeof(T) == 8;
  const int kind = UNI ? (f64 ? PF_PROF_CG_PASS_FP64_PF1 : PF_PROF_CG_PASS_FP32_PF1)
                       : (f64 ? PF_PROF_CG_PASS_FP64 : PF_PROF_CG_PASS_FP32);
  pf::Maps<S::NH, S::NC> m[2];
  for (int cur = 0; cur < 2; ++cur) {
    if constexpr (UNI) {
      const T* h[S::NH] = {K.r[cur], K.v[cur], K.p[cur], A.dinv};
      const T* c[S::NC] = {K.t, x};
      PF_TRY((fill_maps<S::NH, S::NC, T>(g, &m[cur], h, c)));
    } else if constexpr (pf::ca_face_from_gh<T>()) {
      const T* h[S::NH] = {K.r[cur], K.v[cur], K.p[cur], A.dinv, A.gh};
      const T* c[S::NC] = {K.t, x};
      PF_TRY((fill_maps<S::NH, S::NC, T>(g, &m[cur], h, c)));
    } else {
      const T* h[S::NH] = {K.r[cur], K.v[cur], K.p[cur], A.dinv, A.wE, A.wN};
      const T* c[S::NC] = {K.t, x, A.wU};
      PF_TRY((fill_maps<S::NH, S::NC, T>(g, &m[cur], h, c)));
    }
  }
  const T wc = (T)A.wc;
  PF_LAUNCH(g, kind, (pf::launch_cg_pass<T, UNI>(m[0], g->geom, wc, K.r[1], K.v[1], K.p[1], K.t, x, g->part, st, 1,
                                                 g->L)));
  int cur = 1;
  for (;;) {
    for (int i = 0; i < CHUNK; ++i) {
      PF_LAUNCH(g, kind, (pf::launch_cg_pass<T, UNI>(m[cur], g->geom, wc, K.r[1 - cur], K.v[1 - cur], K.p[1 - cur],
                                                     K.t, x, g->part, st, 0, g->L)));
      cur = 1 - cur;
    }
    BicgState s;
    PF_TRY(read_state(g, st, &s));
    if (s.done) {
      *out = s;
      return PF_OK;
    }
  }
}

// Conjugate gradients in place of BiCGSTAB for this operator?
bool use_cg(const pf_solve_opts& o, int op) {
  return o.method == PF_CG_ALL || (o.method == PF_CG_SYMMETRIC && op != PF_OP_PF2);
}

double measure_of(const BicgState& s, int norm) {
  return norm == PF_NORM_REL2 ? sqrt(s.rnorm2 / s.bnorm2) : s.rinf;
}

template <bool UNI>
pf_status solve_fp64(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, double tol_r0,
                     pf_report* rep) {
  const OpArrays<double> A = ops64(g, op);
  const Krylov<double> K = kry64(g);
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x, b, A.dinv, g->geom.np, g->stream));
  PF_TRY(set_state(g, g->st, o.tol, o.norm, o.max_iter, tol_r0));
  PF_TRY(residual<UNI>(g, A, x, b, 1, &K, g->st));  // r0 = b - A x0 (Table 3)
  BicgState s;
  if (use_cg(o, op))
    PF_TRY((iterate_cg<double, UNI>(g, A, x, K, g->st, &s)));
  else
    PF_TRY((iterate<double, UNI>(g, A, x, K, g->st, &s)));
  // true residual of the final iterate (b.b kept from the start)
  BicgState tr;
  PF_TRY(set_state(g, g->st, o.tol, o.norm, 0, tol_r0, 1));
  pf::ResidualExtras ex;
  ex.need_bb = 0;
  ex.need_max = o.norm == PF_NORM_ABSINF;
  PF_TRY(residual<UNI>(g, A, x, b, 0, nullptr, g->st, ex));
  PF_TRY(read_state(g, g->st, &tr));
  rep->status = s.status;
  rep->iterations = s.iter;
  rep->refinements = 0;
  rep->residual = measure_of(tr, o.norm);
  if (trace_level() > 0)
    fprintf(stderr, "[pf] fp64 solve op %d: status %d iters %d residual %.3e\n", op, rep->status, rep->iterations,
            rep->residual);
  return PF_OK;
}

template <bool UNI>
pf_status solve_mixed(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, double tol_r0,
                      pf_report* rep) {
  const OpArrays<double> A = ops64(g, op);
  const OpArrays<float> W = ops32(g, op);
  const Krylov<float> K = kry32(g);
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x, b, A.dinv, g->geom.np, g->stream));
  int iters = 0, ref = 0, status = PF_E_NOCONV;
  BicgState tr{};
  for (;;) {
    // FP64 true residual b - A x and its norms; the same pass starts the FP32 inner solve A d = r from d = 0
    // (r = r~ = (float) r, p = v = t = 0) to relative tolerance inner_tol; an inner solve that stagnates is cut
    // off after INNER_CAP iterations and its correction kept
    const int cap = o.max_iter - iters < INNER_CAP ? o.max_iter - iters : INNER_CAP;
    PF_TRY(set_state(g, g->st, o.tol, o.norm, 0, tol_r0, ref > 0));
    PF_TRY(set_state(g, g->st2, o.inner_tol, PF_NORM_REL2, cap > 0 ? cap : 1));
    pf::ResidualExtras ex;
    ex.need_bb = ref == 0;
    ex.need_max = o.norm == PF_NORM_ABSINF;
    ex.r = K.r[0];
    ex.rt = K.rt;
    ex.p = K.p[0];
    ex.v = K.v[0];
    ex.t = K.t;
    ex.d = g->d32;
    ex.st2 = g->st2;
    PF_TRY(residual<UNI>(g, A, x, b, 0, nullptr, g->st, ex));
    PF_TRY(read_state(g, g->st, &tr));
    if (trace_level() > 0)
      fprintf(stderr, "[pf] mixed op %d refinement %d: true residual %.3e\n", op, ref, measure_of(tr, o.norm));
    if (tr.done) {
      status = PF_OK;
      break;
    }
    if (!isfinite(tr.rnorm2)) {
      status = PF_E_BREAKDOWN;
      break;
    }
    if (ref >= o.max_refine || iters >= o.max_iter) {
      status = PF_E_NOCONV;
      break;
    }
    // a step that can end the refinement stops its inner solve at FINAL_INNER_MARGIN of the target
    const double t2 = final_inner_tol2(o, tr.rnorm2, tr.tol2);
    if (t2 > 0.0) PF_TRY(raise_tol2(g, g->st2, t2, g->stream));
    BicgState s;
    if (use_cg(o, op))
      PF_TRY((iterate_cg<float, UNI>(g, W, g->d32, K, g->st2, &s)));
    else
      PF_TRY((iterate<float, UNI>(g, W, g->d32, K, g->st2, &s)));
    iters += s.iter;
    ++ref;
    if (s.status == PF_E_BREAKDOWN && s.iter == 0) {
      status = PF_E_BREAKDOWN;
      break;
    }
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_add_f32(x, g->d32, g->geom.np, g->stream));  // x += d
  }
  rep->status = status;
  rep->iterations = iters;
  rep->refinements = ref;
  rep->residual = measure_of(tr, o.norm);
  return PF_OK;
}

// Jacobi-preconditioned conjugate gradients in FP64 (the symmetric systems of Section 3): a start kernel,
// then [direction, update] pairs in chunks of CHUNK iterations between reads of the device state, and the
// true residual of the final iterate.
pf_status solve_cg(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, pf_report* rep) {
  const OpArrays<double> A = ops64(g, op);
  const Krylov<double> K = kry64(g);
  const pf::CgOperator C{A.dinv, A.diag, A.wE, A.wN, A.wU, A.wc, A.diagc};
  cudaStream_t s = g->stream;
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x, b, A.dinv, g->geom.np, s));
  PF_TRY(set_state(g, g->st, o.tol, o.norm, o.max_iter));
  PF_LAUNCH(g, PF_PROF_INIT, pf::launch_cg_start(C, g->geom, b, x, K.r[0], K.p[0], g->part, g->st, s));
  BicgState st{};
  int cur = 0;
  // the device state ends the solve by max_iter at the latest; the host bound only guards that
  for (long launched = 0;; launched += CHUNK) {
    PF_TRY(read_state(g, g->st, &st));
    if (st.done) break;
    if (launched > (long)o.max_iter + 2 * CHUNK) {
      st.status = PF_E_NOCONV;
      break;
    }
    for (int i = 0; i < CHUNK; ++i) {
      PF_LAUNCH(g, PF_PROF_CG_DIRECTION,
                pf::launch_cg_direction(C, g->geom, K.r[0], K.p[cur], K.p[1 - cur], K.v[0], g->part, g->st, s));
      PF_LAUNCH(g, PF_PROF_CG_UPDATE, pf::launch_cg_update(C, g->geom, K.p[1 - cur], K.v[0], x, K.r[0], g->part, g->st, s));
      cur = 1 - cur;
    }
  }
  BicgState tr{};
  PF_TRY(set_state(g, g->st2, o.tol, o.norm, 0));
  PF_LAUNCH(g, PF_PROF_RESIDUAL, pf::launch_cg_start(C, g->geom, b, x, K.t, nullptr, g->part, g->st2, s));
  PF_TRY(read_state(g, g->st2, &tr));
  rep->status = st.status;
  rep->iterations = st.iter;
  rep->refinements = 0;
  rep->residual = measure_of(tr, o.norm);
  if (trace_level() > 0)
    fprintf(stderr, "[pf] cg solve op %d: status %d iters %d residual %.3e\n", op, rep->status, rep->iterations,
            rep->residual);
  return PF_OK;
}

// tol_r0 > 0 also accepts ||r||_2 <= tol_r0 ||r0||_2 (r0: the residual of the starting x), the forcing
// term of an inexact outer iteration
pf_status solve_dev(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, pf_report* rep,
                    double tol_r0 = 0.0) {
  NvtxRange range(op == PF_OP_PF1 ? "PF1 solve" : op == PF_OP_PF2 ? "PF2 solve" : "Poisson solve");
  const bool uni = op == PF_OP_PF1;
  if (o.precision == PF_MIXED)
    return uni ? solve_mixed<true>(g, op, b, x, o, tol_r0, rep) : solve_mixed<false>(g, op, b, x, o, tol_r0, rep);
  return uni ? solve_fp64<true>(g, op, b, x, o, tol_r0, rep) : solve_fp64<false>(g, op, b, x, o, tol_r0, rep);
}

pf_status check_opts(const pf_solve_opts& o) {
  if (o.max_iter < 1 || !(o.tol > 0) || (o.norm != PF_NORM_REL2 && o.norm != PF_NORM_ABSINF) ||
      (o.precision != PF_FP64 && o.precision != PF_MIXED) || !(o.inner_tol > 0 && o.inner_tol < 1) ||
      o.max_refine < 1 || o.method < PF_BICGSTAB || o.method > PF_CG_ALL)
    return fail(PF_E_INVAL, "invalid pf_solve_opts");
  return PF_OK;
}

pf_status update_pf2(pf_grid* g) {
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_eps_diag(g->dsum, g->sig, g->solvent, g->geom, g->diag2, g->dinv2, g->dinv2_32, g->stream));
  if (g->filter_on)
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_filter_rows(g->fmask, g->geom, g->dinv2, g->diag2, g->dinv2_32, g->stream));
  return PF_OK;
}

// the filter region's identity rows in the Poisson and PF1 operators (PF2: update_pf2)
pf_status filter_rows_p1(pf_grid* g) {
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_rows(g->fmask, g->geom, g->dinvP, g->diagP, g->dinvP32, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_rows(g->fmask, g->geom, g->dinv1, nullptr, g->dinv1_32, g->stream));
  return PF_OK;
}

// Step a1 on the device from the stored eps, solvent mask and charges: harmonic faces (Eqs. 15-18
// with zero jump) in FP64 and FP32, diagonals and Jacobi scalings of the three operators, the
// trilinear fixed-charge source (Eq. 3).  kappa (PF2) is reset to zero.  Sets g->err when a charge
// lies outside the grid.
pf_status build_operators(pf_grid* g) {
  const long NP = g->geom.np;
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_faces(g->eps, g->geom, g->h, g->wE, g->wN, g->wU, g->dsum, g->gh32, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wE, g->wE32, NP, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wN, g->wN32, NP, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wU, g->wU32, NP, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_eps_diag(g->dsum, nullptr, nullptr, g->geom, g->diagP, g->dinvP, g->dinvP32, g->stream));
  PF_CK(cudaMemsetAsync(g->sig, 0, NP * sizeof(double), g->stream));
  PF_TRY(update_pf2(g));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_pf1_dinv(g->solvent, g->geom, 1.0 / (6.0 * pf1_face(g) + g->eps_s),
                                                  g->dinv1, g->dinv1_32, g->stream));
  if (g->filter_on) PF_TRY(filter_rows_p1(g));
  PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), g->stream));
  if (g->charge_mode == 1) {  // the decomposition's interface right-hand side replaces the spread charges
    PF_CK(cudaMemcpyAsync(g->ffix, g->bif, NP * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    return PF_OK;
  }
  PF_CK(cudaMemsetAsync(g->ffix, 0, NP * sizeof(double), g->stream));
  if (g->nq > 0)
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_spread(g->dch, g->nq, g->origin[0], g->origin[1], g->origin[2], g->h,
                                                  g->lam, g->geom, g->ffix, g->err, g->stream));
  return PF_OK;
}

// compact caller array (host or device) -> padded device array
pf_status pack_in(pf_grid* g, const void* src, int mem, void* dst, int type) {
  const size_t bytes = g->N * (type == 0 ? sizeof(double) : 1);
  const void* from = src;
  if (mem != PF_MEM_DEVICE) {
    PF_CK(cudaMemcpyAsync(g->stage, src, bytes, cudaMemcpyHostToDevice, g->stream));
    from = g->stage;
  }
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_pack(from, dst, g->geom, type, g->stream));
  return PF_OK;
}

// padded device field(s) -> compact caller array (host or device), `count` consecutive fields
pf_status unpack_out(pf_grid* g, const double* src, int count, double* dst, int mem) {
  for (int f = 0; f < count; ++f) {
    double* to = mem == PF_MEM_DEVICE ? dst + (size_t)f * g->N : g->stage;
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_unpack(src + (size_t)f * g->geom.np, to, g->geom, 1, g->stream));
    if (mem != PF_MEM_DEVICE)
      PF_CK(cudaMemcpyAsync(dst + (size_t)f * g->N, g->stage, g->N * sizeof(double), cudaMemcpyDeviceToHost,
                            g->stream));
  }
  return PF_OK;
}

// Starting vectors of the linear solves of the outer iteration (pf_nl_opts.predict).  x holds the last solution
// x_{k-1}; h0 and h1 the two before it (x_{k-2}, x_{k-3}).  The next start is x_{k-1} + c (x_{k-1} - x_{k-2}).
constexpr int PREDICT_THREADS = 256;

// Block partials of d1.d0 and d0.d0 (d1 = x - h0, d0 = h0 - h1) into part[2 b], part[2 b + 1].
__global__ void __launch_bounds__(PREDICT_THREADS) k_predict_dots(const double* __restrict__ x,
                                                                  const double* __restrict__ h0,
                                                                  const double* __restrict__ h1, long n,
                                                                  double* __restrict__ part) {
  __shared__ double sh[2][PREDICT_THREADS / 32];
  double a = 0.0, b = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double p = h0[i];
    const double d1 = x[i] - p, d0 = p - h1[i];
    a = fma(d1, d0, a);
    b = fma(d0, d0, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < PREDICT_THREADS / 32; ++k) {
      sa += sh[0][k];
      sb += sh[1][k];
    }
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

// x <- x + c (x - h0) and hnew <- the old x.  With nparts > 0 every block first sums the nparts block partials of
// k_predict_dots in the same fixed order and takes c = d1.d0 / d0.d0 clamped to [0, 1] (0 when d0 = 0); else
// c = c_fixed, and with c_fixed = 0 x is kept and h0 is not read.
__global__ void __launch_bounds__(PREDICT_THREADS) k_predict(double* __restrict__ x, const double* __restrict__ h0,
                                                             double* __restrict__ hnew, double c_fixed,
                                                             const double* __restrict__ part, int nparts, long n) {
  __shared__ double sh[2][PREDICT_THREADS];
  double c = c_fixed;
  if (nparts > 0) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nparts; k += PREDICT_THREADS) {
      a += part[2 * k];
      b += part[2 * k + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int st = PREDICT_THREADS / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
        sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
      }
      __syncthreads();
    }
    const double num = sh[0][0], den = sh[1][0];
    c = den > 0.0 ? num / den : 0.0;
    c = c > 0.0 ? (c < 1.0 ? c : 1.0) : 0.0;  // also maps a NaN ratio to 0
  }
  const bool extrapolate = c != 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double t = x[i];
    if (extrapolate) x[i] = fma(c, t - h0[i], t);
    hnew[i] = t;
  }
}

// have = solutions of this system so far in this solve (>= 1).  have = 1 only saves x; have = 2 extrapolates with
// c_fallback (the outer updates' ratio); from have = 3 on, with c from the vector's own last two changes.  The
// history pointers rotate, so the newest previous solution is always h0.
pf_status predict(pf_grid* g, double* x, double*& h0, double*& h1, int have, double c_fallback) {
  const long n = g->geom.np;
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long blocks = (n + PREDICT_THREADS - 1) / PREDICT_THREADS;
  if (blocks > 8L * nsm) blocks = 8L * nsm;  // partials: 2 per block, well inside the grid's partials buffer
  cudaStream_t s = g->stream;
  if (have <= 1) {
    PF_LAUNCH(g, PF_PROF_OTHER,
              (k_predict<<<(int)blocks, PREDICT_THREADS, 0, s>>>(x, nullptr, h0, 0.0, nullptr, 0, n),
               cudaGetLastError()));
    return PF_OK;
  }
  int nparts = 0;
  if (have >= 3) {
    PF_LAUNCH(g, PF_PROF_OTHER,
              (k_predict_dots<<<(int)blocks, PREDICT_THREADS, 0, s>>>(x, h0, h1, n, g->part), cudaGetLastError()));
    nparts = (int)blocks;
  }
  PF_LAUNCH(g, PF_PROF_OTHER,
            (k_predict<<<(int)blocks, PREDICT_THREADS, 0, s>>>(x, h0, h1, have >= 3 ? 0.0 : c_fallback, g->part,
                                                                 nparts, n),
             cudaGetLastError()));
  double* t = h0;  // h1 now holds x_{k-1}, h0 x_{k-2}
  h0 = h1;
  h1 = t;
  return PF_OK;
}

__global__ void k_raise_tol2(BicgState* st, double t2) {
  if (blockIdx.x == 0 && threadIdx.x == 0) st->tol2 = fmax(st->tol2, t2);
}

pf_status raise_tol2(pf_grid* g, BicgState* st, double t2, cudaStream_t s) {
  PF_LAUNCH(g, PF_PROF_OTHER, (k_raise_tol2<<<1, 32, 0, s>>>(st, t2), cudaGetLastError()));
  return PF_OK;
}

double final_inner_tol2(const pf_solve_opts& o, double rr, double t2) {
  if (o.norm != PF_NORM_REL2) return 0.0;
  const double f2 = FINAL_INNER_MARGIN * FINAL_INNER_MARGIN * t2;
  return f2 > o.inner_tol * o.inner_tol * rr ? f2 : 0.0;
}

pf_status ensure_predict(pf_grid* g) {
  if (g->xp_psi) return PF_OK;
  PF_TRY(dalloc(g, &g->xp_psi, g->geom.np));
  PF_TRY(dalloc(g, &g->xpp_psi, g->geom.np));
  PF_TRY(dalloc(g, &g->xp_phi, g->geom.np));
  PF_TRY(dalloc(g, &g->xpp_phi, g->geom.np));
  return PF_OK;
}

// Buffers of Anderson acceleration with depth m (kept for later solves on the grid).
pf_status ensure_aa(pf_grid* g, int m) {
  const long NP = g->geom.np;
  if (!g->aa_f) {
    PF_TRY(dalloc(g, &g->aa_f, NP));
    PF_TRY(dalloc(g, &g->aa_fprev, NP));
    PF_TRY(dalloc(g, &g->aa_xprev, NP));
    PF_TRY(dalloc(g, &g->aa_out, 2 * pf::AA_MAX));
  }
  for (; g->aa_alloc < m; ++g->aa_alloc) {
    PF_TRY(dalloc(g, &g->aa_dF[g->aa_alloc], NP));
    PF_TRY(dalloc(g, &g->aa_dX[g->aa_alloc], NP));
  }
  return PF_OK;
}

// Solves (A + reg I) x = b for a small symmetric positive semi-definite A (k <= AA_MAX) by Cholesky;
// false when a pivot is not positive.
bool small_spd_solve(int k, const double (&A)[pf::AA_MAX][pf::AA_MAX], const double* b, double* x) {
  double L[pf::AA_MAX][pf::AA_MAX] = {};
  double tr = 0.0;
  for (int i = 0; i < k; ++i) tr = fmax(tr, A[i][i]);
  const double reg = 1e-10 * (tr > 0 ? tr : 1.0);
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      double sum = A[i][j] + (i == j ? reg : 0.0);
      for (int q = 0; q < j; ++q) sum -= L[i][q] * L[j][q];
      if (i == j) {
        if (!(sum > 0.0)) return false;
        L[i][i] = sqrt(sum);
      } else {
        L[i][j] = sum / L[j][j];
      }
    }
  }
  double y[pf::AA_MAX];
  for (int i = 0; i < k; ++i) {
    double sum = b[i];
    for (int q = 0; q < i; ++q) sum -= L[i][q] * y[q];
    y[i] = sum / L[i][i];
  }
  for (int i = k - 1; i >= 0; --i) {
    double sum = y[i];
    for (int q = i + 1; q < k; ++q) sum -= L[q][i] * x[q];
    x[i] = sum / L[i][i];
  }
  for (int i = 0; i < k; ++i)
    if (!isfinite(x[i])) return false;
  return true;
}

pf_status outer_stage1(pf_grid* g, OuterUpdate& u, int m, double omega) {
  const long NP = g->geom.np;
  cudaStream_t s = g->stream;
  if (m == 0) {
    // relaxation and stop test of Table 4
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_relax(g->phi0, g->phi, omega, NP, g->part, g->ticket, g->delta, s));
  } else {
    // Anderson acceleration of the same map: f = Phi_solve - Phi_0, delta = (1-omega) ||f||_inf is the
    // relaxed update of Table 4; the accelerated update mixes the last m differences of f and Phi_0
    u.slot = u.head;
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_aa_residual(g->phi, g->phi0, g->aa_f, g->aa_fprev, g->aa_xprev, g->aa_dF[u.slot],
                                     g->aa_dX[u.slot], u.kaa >= 1, NP, g->part, g->ticket, g->delta, s));
  }
  PF_CK(cudaMemcpyAsync(g->host_delta, g->delta, sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return PF_OK;
}

double outer_delta(const pf_grid* g, int m, double omega) {
  return m == 0 ? *g->host_delta : (1.0 - omega) * *g->host_delta;
}

pf_status outer_stage2(pf_grid* g, OuterUpdate& u, int m, bool stop) {
  u.dots = false;
  u.cols = pf::AAPtrs{};
  if (m == 0 || stop || u.kaa < 1) return PF_OK;
  u.head = (u.head + 1) % m;
  u.nact = u.nact < m ? u.nact + 1 : m;
  for (int j = 0; j < u.nact; ++j) {  // active slots, oldest first
    u.act[j] = ((u.head - u.nact + j) % m + m) % m;
    u.cols.dF[j] = g->aa_dF[u.act[j]];
    u.cols.dX[j] = g->aa_dX[u.act[j]];
  }
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_aa_dots(u.cols, u.nact, g->aa_dF[u.slot], g->aa_f, g->geom.np, g->part,
                                                 g->ticket, g->aa_out, g->stream));
  PF_CK(cudaMemcpyAsync(g->aa_host, g->aa_out, 2 * pf::AA_MAX * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  u.dots = true;
  return PF_OK;
}

pf_status outer_stage3(pf_grid* g, OuterUpdate& u, int m, double omega, bool stop) {
  if (m == 0) return PF_OK;
  pf::AACoef gam{};
  int k = 0;
  if (u.dots && !stop) {
    const int slot = u.slot, n = u.nact;
    double A[pf::AA_MAX][pf::AA_MAX] = {}, bvec[pf::AA_MAX], x[pf::AA_MAX];
    for (int j = 0; j < n; ++j) u.Gm[slot][u.act[j]] = u.Gm[u.act[j]][slot] = g->aa_host[j];
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) A[i][j] = u.Gm[u.act[i]][u.act[j]];
      bvec[i] = g->aa_host[pf::AA_MAX + i];
    }
    bool ok = small_spd_solve(n, A, bvec, x);
    for (int j = 0; ok && j < n; ++j) ok = fabs(x[j]) < 1e4;
    if (ok) {
      k = n;
      for (int j = 0; j < n; ++j) gam.g[j] = x[j];
    } else {
      u.nact = 0;  // ill-conditioned history: restart with a plain relaxed step
    }
  }
  // at the stop k = 0: the plain relaxed update, so the final iterate is the relaxed one of Table 4
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_aa_update(u.cols, gam, k, 1.0 - omega, g->phi0, g->aa_f, g->geom.np, g->stream));
  ++u.kaa;
  return PF_OK;
}

}  // namespace pfi

// Species constants of Eq. (1) from the caller's species list (Table 1 constants): v_i = 4 pi a_i^3 / 3,
// v0 = the mean volume over all species, p_i = v_i / v0, Gamma^B = 1 - sum_i v_i cB_i, lambda, the thermal
// voltage k_B T / e and the mol/L -> A^-3 factor.  Returns nullptr, or a message when the list is invalid
// (radius <= 0, bulk < 0, Gamma^B <= 0 or a charged bath).
namespace pf {
const char* species_params(int ns, const pf_species* species, double T_K, SpeciesParams* out, double* tv,
                           double* molar_out) {
  if (ns < 1 || ns > PF_MAX_SPECIES || !species) return "need 1..PF_MAX_SPECIES species";
  if (!(T_K > 0)) return "need T > 0";
  const double molar = NAVO * 1e-27;
  double v[PF_MAX_SPECIES], v0 = 0.0, gB = 1.0, q = 0.0, qs = 0.0;
  for (int i = 0; i < ns; ++i) {
    const pf_species& s = species[i];
    if (!(s.radius_A > 0) || !(s.bulk_M >= 0)) return "species need radius > 0 and bulk >= 0";
    v[i] = 4.0 * M_PI * s.radius_A * s.radius_A * s.radius_A / 3.0;
    v0 += v[i];
  }
  v0 /= ns;
  SpeciesParams sp{};
  sp.ns = ns;
  for (int i = 0; i < ns; ++i) {
    const pf_species& s = species[i];
    const double cB = s.bulk_M * molar;
    sp.z[i] = s.z;
    sp.p[i] = v[i] / v0;
    sp.lvc[i] = cB > 0 ? log(v[i] * cB) : -INFINITY;
    sp.lcB[i] = cB > 0 ? log(cB) : -INFINITY;
    sp.inv_v[i] = 1.0 / v[i];
    sp.inv_p[i] = 1.0 / sp.p[i];
    if (cB > 0) sp.lnn += 1.0;
    gB -= v[i] * cB;
    q += s.z * cB;
    qs += fabs((double)s.z) * cB;
  }
  if (!(gB > 0)) return "bulk void fraction Gamma^B <= 0";
  if (fabs(q) > 1e-12 * (qs > 0 ? qs : 1.0)) return "bath is not electroneutral";
  sp.lgB = log(gB);
  sp.lnn = log(1.0 + sp.lnn);  // ln(n + 1) over the species present
  sp.lam = QE * QE / (EPS0 * KB * T_K * 1e-10);
  *out = sp;
  *tv = KB * T_K / QE;
  *molar_out = molar;
  return nullptr;
}
}  // namespace pf

// Sets the message that pf_last_error returns on this thread (used by entry points in other files).
void pf_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }

// Device bytes that pf_create_grid allocates for a grid (used for the serving budget).
size_t pf_internal_grid_bytes(int nx, int ny, int nz, int accel_depth) {
  const pf::Geom g = pf::make_geom(nx, ny, nz);
  // Anderson acceleration adds f, f_prev, x_prev and two history columns per depth; the count includes the four
  // history vectors of the predicted starting vectors (pf_nl_opts.predict, on by default)
  const int aa = accel_depth > 0 ? 3 + 2 * accel_depth : 0;
  const size_t per_node = (36 + aa) * sizeof(double) + pf::MAXSP * sizeof(double) + 18 * sizeof(float) + 1;
  return (size_t)g.np * per_node + (size_t)pf::max_partial_blocks() * pf::NPART * sizeof(double) + 8192;
}

extern "C" {

size_t pf_grid_bytes(int nx, int ny, int nz, int accel_depth) {
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  return pf_internal_grid_bytes(nx, ny, nz, accel_depth < 0 ? 0 : accel_depth);
}

void pf_default_solve_opts(pf_solve_opts* o) {
  if (!o) return;
  o->max_iter = 20000;
  o->tol = 1e-10;
  o->norm = PF_NORM_REL2;
  o->precision = PF_FP64;
  o->inner_tol = 0.1;
  o->max_refine = 64;
  o->method = PF_BICGSTAB;
}

void pf_default_nl_opts(pf_nl_opts* o) {
  if (!o) return;
  o->omega = 0.3;
  o->tol_outer = 1e-9;
  o->max_outer = 500;
  pf_default_solve_opts(&o->lin);
  o->accel_depth = 0;
  o->lin_forcing = 0.0;
  o->warm_start = 0;
  o->predict = 2;
}

const char* pf_last_error(void) { return g_err.c_str(); }

pf_status pf_create_grid(int nx, int ny, int nz, double h_A, const double origin_A[3], void* cuda_stream,
                         pf_grid** out) {
  if (!out) return fail(PF_E_INVAL, "out is NULL");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 3 || !(h_A > 0) || !origin_A)
    return fail(PF_E_INVAL, "grid needs nx, ny >= 2, nz >= 3, h > 0 and an origin");
  if ((double)nx * ny * nz > 2.0e9) return fail(PF_E_INVAL, "grid too large");
  pf_grid* g = new pf_grid();
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->N = (long)nx * ny * nz;
  g->geom = pf::make_geom(nx, ny, nz);
  g->geom.edges = pf::edges_for(nx, ny, nz);
  g->h = h_A;
  for (int a = 0; a < 3; ++a) g->origin[a] = origin_A[a];
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  pf_status s = allocate(g);
  if (s != PF_OK) {
    free_all(g);
    delete g;
    return s;
  }
  g->L.ntiles = pf::tiles_for(nx, ny, nz, pf::ZC, g->geom.edges);
  g->L.stream = g->stream;
  g->L.wait_limit = WAIT_LIMIT;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    free_all(g);
    delete g;
    return cuda_fail(e, "pf_create_grid");
  }
  *out = g;
  return PF_OK;
}

pf_status pf_profile_enable(pf_grid* g, int on) {
  if (!g) return fail(PF_E_INVAL, "grid is NULL");
  prof_resolve(g);
  if (on) {
    g->launches = 0;
    for (int k = 0; k < PF_PROF_KINDS; ++k) {
      g->pcount[k] = 0;
      g->pms[k] = 0.0;
    }
  }
  g->prof_on = on ? 1 : 0;
  return PF_OK;
}

pf_status pf_profile_get(pf_grid* g, pf_profile* out) {
  if (!g || !out) return fail(PF_E_INVAL, "grid and out are required");
  cudaStreamSynchronize(g->stream);
  prof_resolve(g);
  out->launches = g->launches;
  for (int k = 0; k < PF_PROF_KINDS; ++k) {
    out->count[k] = g->pcount[k];
    out->ms[k] = g->pms[k];
  }
  return PF_OK;
}

pf_status pf_destroy_grid(pf_grid* g) {
  if (!g) return PF_OK;
  cudaStreamSynchronize(g->stream);
  free_all(g);
  delete g;
  return PF_OK;
}

pf_status pf_set_coeffs(pf_grid* g, const pf_coeffs* c) {
  if (!g || !c || !c->eps || !c->solvent) return fail(PF_E_INVAL, "grid, coeffs, eps and solvent are required");
  if (c->n_species < 1 || c->n_species > PF_MAX_SPECIES || !c->species)
    return fail(PF_E_INVAL, "need 1..PF_MAX_SPECIES species");
  if (c->n_charges < 0 || (c->n_charges > 0 && !c->charges)) return fail(PF_E_INVAL, "bad charges");
  if (!(c->eps_s > 0) || !(c->lc_A >= 0) || !(c->T_K > 0)) return fail(PF_E_INVAL, "need eps_s > 0, lc >= 0, T > 0");
  double eps_m = 0.0;
  for (long i = 0; i < g->N; ++i) {
    if (!(c->eps[i] > 0) || c->solvent[i] > 1) return fail(PF_E_INVAL, "eps must be > 0 and solvent 0/1");
    if (!c->solvent[i] && eps_m == eps_m) {  // the membrane dielectric, NaN once two values differ
      if (eps_m == 0.0) eps_m = c->eps[i];
      else if (c->eps[i] != eps_m) eps_m = NAN;
    }
  }
  pf::SpeciesParams sp{};
  double tv = 0.0, molar = 0.0;
  if (const char* why = pf::species_params(c->n_species, c->species, c->T_K, &sp, &tv, &molar))
    return fail(PF_E_INVAL, why);
  g->T = c->T_K;
  g->Tv = tv;
  g->lam = sp.lam;
  g->sp = sp;
  g->spd = pf::species_df(sp);
  g->molar = molar;
  g->eps_s = c->eps_s;
  g->lc = c->lc_A;
  g->lo_hat = c->phi_zlo_V / g->Tv;
  g->hi_hat = c->phi_zhi_V / g->Tv;

  PF_TRY(pack_in(g, c->eps, PF_MEM_HOST, g->eps, 0));
  PF_TRY(pack_in(g, c->solvent, PF_MEM_HOST, g->solvent, 1));
  if (g->dch) {
    cudaFreeAsync(g->dch, g->stream);
    g->dch = nullptr;
  }
  g->nq = c->n_charges;
  if (g->nq > 0) {
    PF_CK(cudaMallocAsync(&g->dch, sizeof(double) * 4 * g->nq, g->stream));
    PF_CK(cudaMemcpyAsync(g->dch, c->charges, sizeof(double) * 4 * g->nq, cudaMemcpyHostToDevice, g->stream));
  }
  g->filter_on = false;  // new coefficients: the filter region and the charge treatment must be set again
  g->charge_mode = 0;
  g->eps_m = eps_m;
  PF_TRY(build_operators(g));
  PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  PF_CK(cudaStreamSynchronize(g->stream));
  if (*g->host_err) return fail(PF_E_INVAL, "a fixed charge lies outside the grid");
  g->have_coeffs = true;
  g->have_phi0 = false;
  g->ulast_valid = false;
  g->u32_valid = false;
  return PF_OK;
}

pf_status pf_selftest_wait_timeout(unsigned long long limit_cycles, void* cuda_stream) {
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  int h = -1;
  PF_CK(cudaMallocAsync(&d, sizeof(int), s));
  cudaError_t e = pf::launch_wait_probe(limit_cycles, d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (h == 7) return fail(PF_E_TIMEOUT, "the bounded wait gave up as intended");
  return PF_OK;
}

pf_status pf_set_potential(pf_grid* g, const double* phi_V, int mem) {
  if (!g || !phi_V) return fail(PF_E_INVAL, "grid and phi_V are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  if (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "mem must be PF_MEM_HOST or PF_MEM_DEVICE");
  const long NP = g->geom.np;
  PF_TRY(pack_in(g, phi_V, mem, g->phi0, 0));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->phi0, 1.0 / g->Tv, g->phi0, NP, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_dirichlet(g->phi0, g->lo_hat, g->hi_hat, g->geom, g->stream));
  PF_CK(cudaMemsetAsync(g->psi, 0, NP * sizeof(double), g->stream));
  PF_CK(cudaStreamSynchronize(g->stream));
  g->have_phi0 = true;
  g->ulast_valid = false;
  return PF_OK;
}

pf_status pf_set_kappa(pf_grid* g, const double* kappa, int mem) {
  if (!g || !kappa) return fail(PF_E_INVAL, "grid and kappa are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  PF_TRY(pack_in(g, kappa, mem, g->sig, 0));
  PF_TRY(update_pf2(g));
  PF_CK(cudaStreamSynchronize(g->stream));
  return PF_OK;
}

static pf_status linear_solve_entry(pf_grid* g, int op, const double* b, double* x, int mem,
                                    const pf_solve_opts* opts, pf_report* report, bool cg) {
  if (!g || !b || !x) return fail(PF_E_INVAL, "grid, b and x are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  if (op != PF_OP_POISSON && op != PF_OP_PF1 && op != PF_OP_PF2) return fail(PF_E_INVAL, "unknown operator");
  if (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "mem must be PF_MEM_HOST or PF_MEM_DEVICE");
  pf_solve_opts o;
  if (opts) o = *opts; else pf_default_solve_opts(&o);
  PF_TRY(check_opts(o));
  if (cg && o.precision != PF_FP64) return fail(PF_E_INVAL, "conjugate gradients runs in FP64 only");
  pf_report rep{};
  PF_CK(cudaEventRecord(g->ev0, g->stream));
  PF_TRY(pack_in(g, b, mem, g->bb, 0));
  PF_TRY(pack_in(g, x, mem, g->xb, 0));
  if (cg) {
    NvtxRange r2("CG solve");
    PF_TRY(solve_cg(g, op, g->bb, g->xb, o, &rep));
  } else {
    PF_TRY(solve_dev(g, op, g->bb, g->xb, o, &rep));
  }
  PF_TRY(unpack_out(g, g->xb, 1, x, mem));
  PF_CK(cudaEventRecord(g->ev1, g->stream));
  PF_CK(cudaEventSynchronize(g->ev1));
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
  prof_resolve(g);
  rep.time_ms = ms;
  if (report) *report = rep;
  if (rep.status != PF_OK)
    return fail((pf_status)rep.status, rep.status == PF_E_NOCONV ? "linear solve did not converge"
                                       : rep.status == PF_E_TIMEOUT ? "a device wait timed out"
                                       : cg ? "conjugate gradients breakdown (operator not positive definite)"
                                            : "BiCGSTAB breakdown");
  return PF_OK;
}

pf_status pf_set_charge_mode(pf_grid* g, int mode, pf_report* rep) {
  if (!g) return fail(PF_E_INVAL, "grid is required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  if (mode != PF_CHARGES_SPREAD && mode != PF_CHARGES_DECOMPOSED) return fail(PF_E_INVAL, "bad charge mode");
  if (rep) *rep = pf_report{};
  if (mode == PF_CHARGES_SPREAD) {
    g->charge_mode = 0;
    return PF_OK;
  }
  if (g->nx < 3 || g->ny < 3) return fail(PF_E_INVAL, "the decomposition needs nx, ny >= 3");
  if (!(g->eps_m == g->eps_m)) return fail(PF_E_INVAL, "the decomposition needs a uniform membrane dielectric");
  const long NP = g->geom.np;
  cudaStream_t s = g->stream;
  if (!g->Gdec) {
    PF_TRY(dalloc(g, &g->Gdec, NP));
    PF_TRY(dalloc(g, &g->bif, NP));
    PF_CK(cudaMemsetAsync(g->Gdec, 0, NP * sizeof(double), s));
    PF_CK(cudaMemsetAsync(g->bif, 0, NP * sizeof(double), s));
  }
  PF_CK(cudaEventRecord(g->ev0, s));
  // the phi^L matrix (7 diagonals) and its state live in one stream-ordered block for the call
  unsigned char* blk = nullptr;
  const size_t arr = ((size_t)NP * sizeof(double) + 255) / 256 * 256;
  PF_CK(cudaMallocAsync(reinterpret_cast<void**>(&blk), 7 * arr + 256, s));
  double* A[7];
  for (int d = 0; d < 7; ++d) A[d] = reinterpret_cast<double*>(blk + d * arr);
  pf::DiaState* dst = reinterpret_cast<pf::DiaState*>(blk + 7 * arr);
  const double eps_m = g->eps_m > 0 ? g->eps_m : 1.0;  // no membrane node: G = 0 everywhere
  const pf::DecompArgs a{g->dch, g->nq, g->lam / (4.0 * M_PI * eps_m), g->origin[0], g->origin[1], g->origin[2],
                         g->h, eps_m, g->eps_s, g->solvent, g->geom, g->err};
  const pf::DiaVecs w{g->xb, g->bb, g->r64[0], g->rt64, {g->p64[0], g->p64[1]}, {g->v64[0], g->v64[1]}, g->t64};
  pf_status out = PF_OK;
  pf::DiaState hs{};
  do {
    if (cudaMemsetAsync(g->err, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(g->xb, 0, NP * sizeof(double), s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "memset"); break; }
    if (pf::launch_phiL_rows(a, A, g->bb, s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "phiL rows"); break; }
    if (pf::launch_dia_start(A, w, g->geom, 1e-13, 20000, g->part, dst, s) != cudaSuccess) {
      out = cuda_fail(cudaGetLastError(), "phiL start");
      break;
    }
    int cur = 0;
    static_assert(sizeof(pf::DiaState) <= 512, "the state fits the pinned block");
    pf::DiaState* hp = reinterpret_cast<pf::DiaState*>(g->host_st);
    for (long launched = 0;; launched += CHUNK) {
      if (cudaMemcpyAsync(hp, dst, sizeof(pf::DiaState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "phiL state"); break; }
      hs = *hp;
      if (hs.done || launched > 20000 + 2 * CHUNK) break;
      for (int i = 0; i < CHUNK && out == PF_OK; ++i) {
        if (pf::launch_dia_iteration(A, w, cur, g->geom, g->part, dst, s) != cudaSuccess)
          out = cuda_fail(cudaGetLastError(), "phiL iteration");
        cur = 1 - cur;
      }
      if (out != PF_OK) break;
      g->launches += 3 * CHUNK;
    }
    if (out != PF_OK) break;
    if (!hs.done || hs.status != 0) {
      out = fail(hs.status == 4 ? PF_E_BREAKDOWN : PF_E_NOCONV, "the phi^L solve of the decomposition failed");
      break;
    }
    if (pf::launch_decomp_G(a, g->xb, g->Gdec, s) != cudaSuccess ||
        pf::launch_decomp_bif(a, g->xb, g->bif, s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "G / bif"); break; }
    if (cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventRecord(g->ev1, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      out = cuda_fail(cudaGetLastError(), "decomposition");
      break;
    }
    if (*g->host_err)
      out = fail(PF_E_INVAL, *g->host_err == 1 ? "the decomposition needs every charge off the nodes"
                                               : "the decomposition needs each side node to match its mirror partner");
  } while (0);
  cudaFreeAsync(blk, s);
  if (out != PF_OK) return out;
  g->charge_mode = 1;
  if (rep) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    rep->status = PF_OK;
    rep->iterations = hs.iter;
    rep->residual = sqrt(hs.rnorm2 / hs.bnorm2);
    rep->time_ms = ms;
  }
  return PF_OK;
}

pf_status pf_get_decomposition(pf_grid* g, double* G_V, double* b_if, int mem) {
  if (!g) return fail(PF_E_INVAL, "grid is required");
  if (g->charge_mode != 1) return fail(PF_E_INVAL, "pf_set_charge_mode(PF_CHARGES_DECOMPOSED) must come first");
  if (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "bad mem");
  if (G_V) {
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->Gdec, g->Tv, g->phi, g->geom.np, g->stream));
    PF_TRY(unpack_out(g, g->phi, 1, G_V, mem));
  }
  if (b_if) PF_TRY(unpack_out(g, g->bif, 1, b_if, mem));
  PF_CK(cudaStreamSynchronize(g->stream));
  return PF_OK;
}

pf_status pf_set_filter_sites(pf_grid* g, const pf_sites* st, double* site_phi_V, double* site_S) {
  if (!g || !st) return fail(PF_E_INVAL, "grid and sites are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  const int n = st->n_sites;
  if (n < 1 || n > 65535 || !st->center_A || !st->radius_A || !st->q_ion || !st->occupied || !st->ion_radius_A ||
      !(st->eps_b > 0) || !(st->eps_p > 0) || !(st->map_radius_A >= 0) || !(st->v_sites_A3 > 0))
    return fail(PF_E_INVAL, "pf_set_filter_sites: bad site description");
  std::vector<double> packed(8 * (size_t)n);
  for (int b = 0; b < n; ++b) {
    if (!(st->radius_A[b] > 0) || !(st->ion_radius_A[b] > 0) || (st->occupied[b] != 0 && st->occupied[b] != 1))
      return fail(PF_E_INVAL, "pf_set_filter_sites: radii must be > 0 and occupied 0 or 1");
    double* q = &packed[8 * (size_t)b];
    q[0] = st->center_A[3 * b];
    q[1] = st->center_A[3 * b + 1];
    q[2] = st->center_A[3 * b + 2];
    q[3] = st->radius_A[b];
    q[4] = st->q_ion[b];
    q[5] = st->occupied[b];
    q[6] = st->ion_radius_A[b];
    q[7] = 0.0;
  }
  cudaStream_t s = g->stream;
  // site table, potentials, S and the error flag in one small stream-ordered block
  unsigned char* blk = nullptr;
  const size_t tb = packed.size() * sizeof(double), pb = (size_t)n * sizeof(double);
  PF_CK(cudaMallocAsync(reinterpret_cast<void**>(&blk), tb + pb + 2 * sizeof(double), s));
  double* dsite = reinterpret_cast<double*>(blk);
  double* dphi = reinterpret_cast<double*>(blk + tb);
  double* dS = reinterpret_cast<double*>(blk + tb + pb);
  int* derr = reinterpret_cast<int*>(blk + tb + pb + sizeof(double));
  pf_status out = PF_OK;
  std::vector<double> hphi(n);
  double hS = 0.0;
  int herr = 0;
  do {
    if (cudaMemcpyAsync(dsite, packed.data(), tb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(derr, 0, sizeof(int), s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "site copy"); break; }
    if (pf::launch_site_potentials(dsite, n, g->dch, g->nq, st->eps_b, st->eps_p, g->lam, st->v_sites_A3,
                                   g->sp.lgB, dphi, dS, derr, s) != cudaSuccess) {
      out = cuda_fail(cudaGetLastError(), "launch_site_potentials");
      break;
    }
    if (cudaMemcpyAsync(hphi.data(), dphi, pb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hS, dS, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "site results"); break; }
    if (herr) {
      out = fail(PF_E_INVAL, herr == 1 ? "pf_set_filter_sites: a site point coincides with a charge or a site centre"
                                       : "pf_set_filter_sites: the ions fill v_sites_A3");
      break;
    }
    // the region: drop a previous one, then map the sites to the solvent nodes of their spheres
    if (g->filter_on) {
      g->filter_on = false;
      out = build_operators(g);
      if (out != PF_OK) break;
    }
    const long NP = g->geom.np;
    if (!g->fmask) {
      if ((out = dalloc(g, &g->fmask, NP)) != PF_OK) break;
      if ((out = dalloc(g, &g->fval, NP)) != PF_OK) break;
    }
    if (cudaMemsetAsync(g->fmask, 0, NP, s) != cudaSuccess) { out = cuda_fail(cudaGetLastError(), "fmask"); break; }
    if (pf::launch_site_map(dsite, n, dphi, g->solvent, g->geom, g->origin[0], g->origin[1], g->origin[2], g->h,
                            st->map_radius_A, g->fmask, g->fval, s) != cudaSuccess) {
      out = cuda_fail(cudaGetLastError(), "launch_site_map");
      break;
    }
    g->filter_on = true;
    if ((out = filter_rows_p1(g)) != PF_OK) break;
    if (pf::launch_filter_rows(g->fmask, g->geom, g->dinv2, g->diag2, g->dinv2_32, s) != cudaSuccess)
      out = cuda_fail(cudaGetLastError(), "launch_filter_rows");
  } while (0);
  cudaFreeAsync(blk, s);
  if (out != PF_OK) return out;
  if (site_phi_V)
    for (int b = 0; b < n; ++b) site_phi_V[b] = hphi[b] * g->Tv;
  if (site_S) *site_S = hS;
  return PF_OK;
}

pf_status pf_set_filter(pf_grid* g, const uint8_t* fixed, const double* phi_V, int mem) {
  if (!g) return fail(PF_E_INVAL, "grid is required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  if (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "mem must be PF_MEM_HOST or PF_MEM_DEVICE");
  if (fixed && !phi_V) return fail(PF_E_INVAL, "phi_V is required with a filter mask");
  if (fixed && mem == PF_MEM_HOST)
    for (long i = 0; i < g->N; ++i)
      if (fixed[i] > 1) return fail(PF_E_INVAL, "fixed must be 0 or 1");
  if (g->filter_on) {  // drop the previous region: rebuild the operators without its identity rows
    g->filter_on = false;
    PF_TRY(build_operators(g));
  }
  if (!fixed) return PF_OK;
  const long NP = g->geom.np;
  if (!g->fmask) {
    PF_TRY(dalloc(g, &g->fmask, NP));
    PF_TRY(dalloc(g, &g->fval, NP));
  }
  PF_CK(cudaMemsetAsync(g->fmask, 0, NP, g->stream));
  PF_TRY(pack_in(g, fixed, mem, g->fmask, 1));
  PF_TRY(pack_in(g, phi_V, mem, g->fval, 0));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->fval, 1.0 / g->Tv, g->fval, NP, g->stream));
  g->filter_on = true;
  PF_TRY(filter_rows_p1(g));
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_filter_rows(g->fmask, g->geom, g->dinv2, g->diag2, g->dinv2_32, g->stream));
  return PF_OK;
}

pf_status pf_linear_solve(pf_grid* g, int op, const double* b, double* x, int mem, const pf_solve_opts* opts,
                          pf_report* report) {
  NvtxRange range("pf_linear_solve");
  return linear_solve_entry(g, op, b, x, mem, opts, report, false);
}

pf_status pf_linear_solve_cg(pf_grid* g, int op, const double* b, double* x, int mem, const pf_solve_opts* opts,
                             pf_report* report) {
  NvtxRange range("pf_linear_solve_cg");
  return linear_solve_entry(g, op, b, x, mem, opts, report, true);
}

pf_status pf_nonlinear_solve(pf_grid* g, const pf_nl_opts* opts, pf_result* res) {
  NvtxRange range("pf_nonlinear_solve");
  if (!g || !res) return fail(PF_E_INVAL, "grid and result are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  pf_nl_opts o;
  if (opts) o = *opts; else pf_default_nl_opts(&o);
  PF_TRY(check_opts(o.lin));
  if (!(o.omega >= 0 && o.omega < 1) || !(o.tol_outer > 0) || o.max_outer < 1 || o.accel_depth < 0 ||
      o.accel_depth > pf::AA_MAX || !(o.lin_forcing >= 0))
    return fail(PF_E_INVAL, "invalid pf_nl_opts");
  if (o.warm_start != 0 && o.warm_start != 1) return fail(PF_E_INVAL, "invalid pf_nl_opts");
  if (o.predict < 0 || o.predict > 2) return fail(PF_E_INVAL, "invalid pf_nl_opts.predict");
  if (o.warm_start && !g->have_phi0)
    return fail(PF_E_INVAL, "warm_start needs a potential on the grid (a previous solve or pf_set_potential)");
  const int m = o.accel_depth;
  if (m > 0) PF_TRY(ensure_aa(g, m));
  if (o.predict) PF_TRY(ensure_predict(g));
  if (res->mem != PF_MEM_HOST && res->mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "bad result mem");
  const pf::Geom& G = g->geom;
  const long NP = G.np;
  cudaStream_t s = g->stream;
  PF_CK(cudaEventRecord(g->ev0, s));
  res->status = PF_OK;
  res->outer_iters = 0;
  res->lin_iters_total = 0;
  res->lin_iters_first = 0;
  res->delta = 0.0;
  pf_status st = PF_OK;
  pf_report rep{};
  // step a1: operators and fixed-charge source from the device-resident coefficients
  PF_TRY(build_operators(g));
  const bool warm = o.warm_start != 0;
  const bool fermi_warm = warm && g->ulast_valid;
  const bool mixed = o.lin.precision == PF_MIXED;
  if (!warm) {
    // initial potential (Table 4): PF2 with rho' = Psi = 0 -> Phi_0
    PF_CK(cudaMemsetAsync(g->phi0, 0, NP * sizeof(double), s));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_dirichlet(g->phi0, g->lo_hat, g->hi_hat, G, s));
    PF_CK(cudaMemsetAsync(g->psi, 0, NP * sizeof(double), s));
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_pf2_rhs(g->psi, g->solvent, g->ffix, g->eps_s, g->lo_hat, g->hi_hat, G, g->b2, s));
    if (g->filter_on) PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_values(g->fmask, g->fval, G, g->b2, s));
    PF_TRY(solve_dev(g, PF_OP_POISSON, g->b2, g->phi0, o.lin, &rep));
    res->lin_iters_first = rep.iterations;
    res->lin_iters_total += rep.iterations;
    if (rep.status != PF_OK) st = (pf_status)rep.status;
  }
  OuterUpdate U;
  double delta_prev = 1.0, delta_prev2 = 0.0;
  for (int outer = 1; st == PF_OK && outer <= o.max_outer; ++outer) {
    // starting vectors (pf_nl_opts.predict): from the third outer iteration on, the last solution extrapolated
    // along its last change, with c = delta_{k-1} / delta_{k-2} while the outer updates shrink (predict = 1, and
    // predict = 2 in the third), and with c from the vector's own last two changes from the fourth on (predict = 2)
    const int have = outer - 1;  // PF1 / PF2 solutions of this solve so far
    const int pred_have = o.predict == 1 && have > 2 ? 2 : have;
    const double c_pred =
        (o.predict && have >= 2 && delta_prev2 > 0.0 && delta_prev < delta_prev2) ? delta_prev / delta_prev2 : 0.0;
    // forcing term: the linear solves of this outer iteration stop at eta ||r0|| (r0: the residual of the warm
    // start, which shrinks with the outer update) or at lin.tol ||b||, whichever is reached first
    double eta = 0.0;
    if (o.lin_forcing > 0) eta = outer == 1 ? 1e-2 : fmin(1e-2, o.lin_forcing * delta_prev);
    const pf_solve_opts& lo = o.lin;
    // Eq. (1) at Phi_0 -> b_PF1 = -lambda rho, kappa, PF2 right-hand-side part (Table 4)
    PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    if (mixed)  // the in-loop step of the mixed path in double-float on the FP32 pipes
      PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi_df(g->phi0, g->solvent, g->ffix, g->spd, G, g->b1, g->sig, g->c2,
                                                      g->ulast32, outer > 1 || (warm && g->u32_valid), g->err, s));
    else
      PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, G, g->b1, g->sig, g->c2,
                                                   nullptr, nullptr, nullptr, g->ulast, outer > 1 || fermi_warm,
                                                   g->err, s));
    if (g->filter_on) PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_zero(g->fmask, G, g->b1, 1, s));  // Psi = 0
    PF_TRY(update_pf2(g));
    if (o.predict && have >= 1) PF_TRY(predict(g, g->psi, g->xp_psi, g->xpp_psi, pred_have, c_pred));
    PF_TRY(solve_dev(g, PF_OP_PF1, g->b1, g->psi, lo, &rep, eta));  // Eq. (12)
    res->lin_iters_total += rep.iterations;
    if (rep.status != PF_OK) { st = (pf_status)rep.status; break; }
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_pf2_rhs(g->psi, g->solvent, g->c2, g->eps_s, g->lo_hat, g->hi_hat, G, g->b2, s));
    if (g->filter_on) PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_values(g->fmask, g->fval, G, g->b2, s));
    if (o.predict && have >= 1)
      PF_TRY(predict(g, g->phi, g->xp_phi, g->xpp_phi, pred_have, c_pred));  // from the previous PF2 solutions
    else
      PF_CK(cudaMemcpyAsync(g->phi, g->phi0, NP * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PF_TRY(solve_dev(g, PF_OP_PF2, g->b2, g->phi, lo, &rep, eta));  // Eq. (13)
    res->lin_iters_total += rep.iterations;
    if (rep.status != PF_OK) { st = (pf_status)rep.status; break; }
    PF_TRY(outer_stage1(g, U, m, o.omega));
    PF_CK(cudaStreamSynchronize(s));
    const double delta = outer_delta(g, m, o.omega);
    const bool stop = delta <= o.tol_outer;
    PF_TRY(outer_stage2(g, U, m, stop));
    if (U.dots) PF_CK(cudaStreamSynchronize(s));
    PF_TRY(outer_stage3(g, U, m, o.omega, stop));
    if (*g->host_err) { st = PF_E_GAMMA; break; }
    res->outer_iters = outer;
    res->delta = delta;
    delta_prev2 = delta_prev;
    delta_prev = delta;
    if (trace_level() > 0)
      fprintf(stderr, "[pf] outer %d delta %.6e lin_total %d eta %.1e\n", outer, res->delta, res->lin_iters_total,
              eta);
    if (res->delta <= o.tol_outer) break;
    if (outer == o.max_outer) st = PF_E_NOCONV;
  }
  // outputs at the final potential
  PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
  // (FP64 in both precisions; after double-float steps it starts from their FP32 roots)
  const bool df_ran = mixed && res->outer_iters > 0;
  PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, G, nullptr, nullptr, nullptr,
                                               g->Cbuf, g->Sbuf, g->Gbuf, g->ulast, res->outer_iters > 0 || fermi_warm,
                                               g->err, s, df_ran ? g->ulast32 : nullptr));
  if (g->filter_on) {  // no continuum concentrations on the filter region
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_zero(g->fmask, G, g->Cbuf, g->sp.ns, s));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_zero(g->fmask, G, g->Sbuf, 1, s));
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_filter_zero(g->fmask, G, g->Gbuf, 1, s));
  }
  if (res->phi_V) {  // phi = phi~ + G in the membrane when the charges are decomposed (Eq. 5)
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_add_scale(g->phi0, g->charge_mode == 1 ? g->Gdec : nullptr, g->Tv, g->phi, NP, s));
    PF_TRY(unpack_out(g, g->phi, 1, res->phi_V, res->mem));
  }
  if (res->C_M) {
    const long nc = NP * g->sp.ns;
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->Cbuf, 1.0 / g->molar, g->Cbuf, nc, s));
    PF_TRY(unpack_out(g, g->Cbuf, g->sp.ns, res->C_M, res->mem));
  }
  if (res->S) PF_TRY(unpack_out(g, g->Sbuf, 1, res->S, res->mem));
  if (res->Gamma) PF_TRY(unpack_out(g, g->Gbuf, 1, res->Gamma, res->mem));
  if (res->Psi) PF_TRY(unpack_out(g, g->psi, 1, res->Psi, res->mem));
  PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PF_CK(cudaEventRecord(g->ev1, s));
  PF_CK(cudaEventSynchronize(g->ev1));
  if (*g->host_err && st == PF_OK) st = PF_E_GAMMA;
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
  prof_resolve(g);
  res->time_ms = ms;
  res->status = st;
  g->have_phi0 = true;
  g->ulast_valid = true;
  if (df_ran) g->u32_valid = true;
  if (st != PF_OK) return fail(st, "nonlinear solve ended with status " + std::to_string((int)st));
  return PF_OK;
}

}  // extern "C"
