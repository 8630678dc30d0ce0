// pf_api.cu -- the C ABI of include/pf_gb300.h: grid state, coefficient setup, and the host
// control of the device solvers (Table 3 linear solver, Table 4 nonlinear solver, FP64 iterative
// refinement around FP32 BiCGSTAB).  Every arithmetic step runs in the kernels of pf_kernels.cu;
// this file only allocates, launches, and reads back the few scalars that steer the iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/pf_gb300.h"
#include "pf_internal.cuh"

using pf::BicgState;
using pf::OpView;

namespace {

thread_local std::string g_err;

// Table 1 constants
constexpr double KB = 1.38e-23;        // J/K
constexpr double QE = 1.602e-19;       // C
constexpr double EPS0 = 8.85e-12;      // F/m (8.85e-14 F/cm)
constexpr double NAVO = 6.02214076e23; // 1/mol (SI value; the paper does not print it)

pf_status fail(pf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

pf_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return PF_E_CUDA;
}

#define PF_CK(call)                                        \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

#define PF_TRY(call)                    \
  do {                                  \
    pf_status s_ = (call);              \
    if (s_ != PF_OK) return s_;         \
  } while (0)

constexpr int CHUNK = 8;  // BiCGSTAB iterations launched between two host checks of the done flag
constexpr int INNER_CAP = 1000;  // FP32 iterations per refinement step at most
constexpr int PROF_SLOTS = 64;  // timed launches between two resolutions of the profiling events

}  // namespace

struct pf_grid {
  int nx = 0, ny = 0, nz = 0;
  long N = 0;
  double h = 1.0, origin[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  pf::Launch L{};
  bool have_coeffs = false;
  // problem constants
  double eps_s = 78.5, lc = 0.0, T = 298.15, Tv = 0.0, lam = 0.0, lo_hat = 0.0, hi_hat = 0.0, molar = 0.0;
  pf::SpeciesParams sp{};
  // device arrays
  std::vector<void*> allocs;
  double *eps = nullptr, *wE = nullptr, *wN = nullptr, *wU = nullptr, *dsum = nullptr, *ffix = nullptr;
  uint8_t* solvent = nullptr;
  double *diagP = nullptr, *dinvP = nullptr, *diag2 = nullptr, *dinv2 = nullptr, *sig = nullptr, *dinv1 = nullptr;
  float *wE32 = nullptr, *wN32 = nullptr, *wU32 = nullptr, *dinvP32 = nullptr, *dinv2_32 = nullptr,
        *dinv1_32 = nullptr;
  double *r64[2] = {nullptr, nullptr}, *p64[2] = {nullptr, nullptr}, *v64[2] = {nullptr, nullptr};
  double *rt64 = nullptr, *t64 = nullptr;
  float *r32[2] = {nullptr, nullptr}, *p32[2] = {nullptr, nullptr}, *v32[2] = {nullptr, nullptr};
  float *rt32 = nullptr, *t32 = nullptr, *d32 = nullptr, *b32 = nullptr;
  double *xb = nullptr, *bb = nullptr;
  double *phi0 = nullptr, *phi = nullptr, *psi = nullptr, *b1 = nullptr, *c2 = nullptr, *b2 = nullptr;
  double *Cbuf = nullptr, *Sbuf = nullptr, *Gbuf = nullptr;
  double* part = nullptr;
  double* dch = nullptr;     // fixed charges (x, y, z, q) on the device
  int nq = 0;
  BicgState* st = nullptr;   // FP64 solve / refinement state
  BicgState* st2 = nullptr;  // FP32 inner solve state
  BicgState* host_st = nullptr;  // pinned mirror
  int* err = nullptr;        // device error flag
  int* host_err = nullptr;   // pinned
  double* delta = nullptr;
  unsigned int* ticket = nullptr;
  double* host_delta = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // profiling: event pairs around launches, resolved at the next host synchronisation
  int prof_on = 0;
  long long launches = 0;
  long long pcount[PF_PROF_KINDS] = {};
  double pms[PF_PROF_KINDS] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<int> pkind;
  int np = 0;
};

namespace {

template <typename T>
pf_status dalloc(pf_grid* g, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PF_E_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed: " +
                              cudaGetErrorString(e));
  }
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return PF_OK;
}

void free_all(pf_grid* g) {
  if (g->dch) cudaFree(g->dch);
  g->dch = nullptr;
  for (cudaEvent_t e : g->pool) cudaEventDestroy(e);
  g->pool.clear();
  for (void* q : g->allocs) cudaFree(q);
  g->allocs.clear();
  if (g->host_st) cudaFreeHost(g->host_st);
  if (g->host_err) cudaFreeHost(g->host_err);
  if (g->host_delta) cudaFreeHost(g->host_delta);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  g->host_st = nullptr;
  g->host_err = nullptr;
  g->host_delta = nullptr;
}

pf_status allocate(pf_grid* g) {
  const long N = g->N;
  double** d64[] = {&g->eps, &g->wE, &g->wN, &g->wU, &g->dsum, &g->ffix, &g->diagP, &g->dinvP, &g->diag2,
                    &g->dinv2, &g->sig, &g->dinv1, &g->r64[0], &g->r64[1], &g->p64[0], &g->p64[1], &g->v64[0],
                    &g->v64[1], &g->rt64, &g->t64, &g->xb, &g->bb, &g->phi0, &g->phi, &g->psi, &g->b1,
                    &g->c2, &g->b2, &g->Sbuf, &g->Gbuf};
  for (double** p : d64) PF_TRY(dalloc(g, p, N));
  PF_TRY(dalloc(g, &g->Cbuf, (size_t)N * pf::MAXSP));
  float** d32[] = {&g->wE32, &g->wN32, &g->wU32, &g->dinvP32, &g->dinv2_32, &g->dinv1_32, &g->r32[0], &g->r32[1],
                   &g->p32[0], &g->p32[1], &g->v32[0], &g->v32[1], &g->rt32, &g->t32, &g->d32, &g->b32};
  for (float** p : d32) PF_TRY(dalloc(g, p, N));
  PF_TRY(dalloc(g, &g->solvent, N));
  PF_TRY(dalloc(g, &g->part, (size_t)pf::max_partial_blocks() * pf::NPART));
  PF_TRY(dalloc(g, &g->st, 1));
  PF_TRY(dalloc(g, &g->st2, 1));
  PF_TRY(dalloc(g, &g->err, 1));
  PF_TRY(dalloc(g, &g->delta, 1));
  PF_TRY(dalloc(g, &g->ticket, 1));
  PF_CK(cudaMallocHost(&g->host_st, sizeof(BicgState)));
  PF_CK(cudaMallocHost(&g->host_err, sizeof(int)));
  PF_CK(cudaMallocHost(&g->host_delta, sizeof(double)));
  // Krylov vectors stay zero on the Dirichlet planes, which no stencil kernel writes
  for (double* p : {g->r64[0], g->r64[1], g->p64[0], g->p64[1], g->v64[0], g->v64[1], g->rt64, g->t64})
    PF_CK(cudaMemsetAsync(p, 0, N * sizeof(double), g->stream));
  for (float* p : {g->r32[0], g->r32[1], g->p32[0], g->p32[1], g->v32[0], g->v32[1], g->rt32, g->t32, g->d32, g->b32})
    PF_CK(cudaMemsetAsync(p, 0, N * sizeof(float), g->stream));
  PF_CK(cudaMemsetAsync(g->st, 0, sizeof(BicgState), g->stream));
  PF_CK(cudaMemsetAsync(g->st2, 0, sizeof(BicgState), g->stream));
  PF_CK(cudaMemsetAsync(g->ticket, 0, sizeof(unsigned int), g->stream));
  PF_CK(cudaMemsetAsync(g->sig, 0, N * sizeof(double), g->stream));
  PF_CK(cudaEventCreate(&g->ev0));
  PF_CK(cudaEventCreate(&g->ev1));
  g->pool.resize(2 * PROF_SLOTS, nullptr);
  g->pkind.resize(PROF_SLOTS, 0);
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

void prof_resolve(pf_grid* g) {
  if (g->np == 0) return;
  if (cudaEventSynchronize(g->pool[2 * (g->np - 1) + 1]) == cudaSuccess) {
    for (int i = 0; i < g->np; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g->pool[2 * i], g->pool[2 * i + 1]) == cudaSuccess) {
        g->pms[g->pkind[i]] += ms;
        g->pcount[g->pkind[i]] += 1;
      }
    }
  }
  cudaGetLastError();
  g->np = 0;
}

int prof_begin(pf_grid* g, int n_launches) {
  g->launches += n_launches;
  if (!g->prof_on) return -1;
  if (g->np == PROF_SLOTS) prof_resolve(g);
  cudaEventRecord(g->pool[2 * g->np], g->stream);
  return g->np;
}

void prof_end(pf_grid* g, int slot, int kind) {
  if (slot < 0) return;
  cudaEventRecord(g->pool[2 * slot + 1], g->stream);
  g->pkind[slot] = kind;
  g->np = slot + 1;
}

#define PF_LAUNCH(g, kind, call)                  \
  do {                                            \
    const int slot_ = prof_begin((g), 1);         \
    PF_CK(call);                                  \
    prof_end((g), slot_, (kind));                 \
  } while (0)

// ---- operator views -----------------------------------------------------------------------
OpView<double> view64(const pf_grid* g, int op) {
  OpView<double> v{};
  v.nx = g->nx;
  v.ny = g->ny;
  v.nz = g->nz;
  if (op == PF_OP_PF1) {
    v.dinv = g->dinv1;
    v.wc = g->eps_s * g->lc * g->lc / (g->h * g->h);
    v.diagc = 6.0 * v.wc + g->eps_s;
  } else {
    v.wE = g->wE;
    v.wN = g->wN;
    v.wU = g->wU;
    v.dinv = op == PF_OP_PF2 ? g->dinv2 : g->dinvP;
    v.diag = op == PF_OP_PF2 ? g->diag2 : g->diagP;
  }
  return v;
}

OpView<float> view32(const pf_grid* g, int op) {
  OpView<float> v{};
  v.nx = g->nx;
  v.ny = g->ny;
  v.nz = g->nz;
  if (op == PF_OP_PF1) {
    v.dinv = g->dinv1_32;
    const double wc = g->eps_s * g->lc * g->lc / (g->h * g->h);
    v.wc = (float)wc;
    v.diagc = 6.0 * wc + g->eps_s;
  } else {
    v.wE = g->wE32;
    v.wN = g->wN32;
    v.wU = g->wU32;
    v.dinv = op == PF_OP_PF2 ? g->dinv2_32 : g->dinvP32;
  }
  return v;
}

pf_status set_state(pf_grid* g, BicgState* dst, double tol, int norm, int max_iter) {
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_state(dst, tol, norm, max_iter, g->stream));
  return PF_OK;
}

pf_status read_state(pf_grid* g, const BicgState* src, BicgState* out) {
  PF_CK(cudaMemcpyAsync(g->host_st, src, sizeof(BicgState), cudaMemcpyDeviceToHost, g->stream));
  PF_CK(cudaStreamSynchronize(g->stream));
  *out = *g->host_st;
  prof_resolve(g);
  return PF_OK;
}

// Runs BiCGSTAB iterations (init, prime, then [B, CA] pairs in chunks) on operator `op` in precision T,
// with the initial residual from x (or x = 0).  Returns the final device state in *out.
template <typename T, bool UNI>
pf_status run_bicgstab(pf_grid* g, const OpView<T>& op, T* x, bool x_zero, const T* b, T* const r[2], T* const p[2],
                       T* const v[2], T* rt, T* t, BicgState* st, BicgState* out) {
  const pf::Launch& L = g->L;
  const bool f64 = sizeof(T) == 8;
  const int kb = UNI ? (f64 ? PF_PROF_B_FP64_PF1 : PF_PROF_B_FP32_PF1) : (f64 ? PF_PROF_B_FP64 : PF_PROF_B_FP32);
  const int kca = UNI ? (f64 ? PF_PROF_CA_FP64_PF1 : PF_PROF_CA_FP32_PF1) : (f64 ? PF_PROF_CA_FP64 : PF_PROF_CA_FP32);
  PF_LAUNCH(g, PF_PROF_INIT, (pf::launch_init<T, UNI>(op, x, x_zero, b, r[0], rt, p[0], v[0], t, g->part, st, L)));
  PF_LAUNCH(g, kca, (pf::launch_phase_ca<T, UNI>(op, r[0], v[0], p[0], t, rt, x, r[1], p[1], v[1], g->part, st, 1, L)));
  int cur = 1;
  for (;;) {
    for (int i = 0; i < CHUNK; ++i) {
      PF_LAUNCH(g, kb, (pf::launch_phase_b<T, UNI>(op, r[cur], v[cur], rt, t, g->part, st, L)));
      PF_LAUNCH(g, kca, (pf::launch_phase_ca<T, UNI>(op, r[cur], v[cur], p[cur], t, rt, x, r[1 - cur], p[1 - cur],
                                                    v[1 - cur], g->part, st, 0, L)));
      cur = 1 - cur;
    }
    BicgState s;
    PF_TRY(read_state(g, st, &s));
    if (trace_level() > 1)
      fprintf(stderr, "[pf] %s it %d rel %.3e rho %.3e alpha %.3e omega %.3e done %d status %d\n",
              sizeof(T) == 8 ? "fp64" : "fp32", s.iter, sqrt(s.rnorm2 / (s.bnorm2 > 0 ? s.bnorm2 : 1.0)), s.rho,
              s.alpha, s.omega, s.done, s.status);
    if (s.done) {
      *out = s;
      return PF_OK;
    }
  }
}

// True FP64 residual of x: fills st (rnorm2, rinf, bnorm2, done) and writes (float)(b - A x) to b32.
template <bool UNI>
pf_status true_residual(pf_grid* g, const OpView<double>& op, double* x, const float* d, const double* b,
                        double tol, int norm, BicgState* out) {
  PF_TRY(set_state(g, g->st, tol, norm, 0));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(b, g->nx, g->ny, g->nz, g->st, g->stream));
  {
    const int slot = prof_begin(g, d ? 2 : 1);
    PF_CK((pf::launch_refine<UNI>(op, x, d, b, g->b32, g->part, g->st, g->L)));
    prof_end(g, slot, PF_PROF_RESIDUAL);
  }
  return read_state(g, g->st, out);
}

double measure_of(const BicgState& s, int norm) {
  return norm == PF_NORM_REL2 ? sqrt(s.rnorm2 / s.bnorm2) : s.rinf;
}

template <bool UNI>
pf_status solve_fp64(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, pf_report* rep) {
  const OpView<double> V = view64(g, op);
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x, b, V.dinv, g->N, g->stream));
  PF_TRY(set_state(g, g->st, o.tol, o.norm, o.max_iter));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_plane_bb(b, g->nx, g->ny, g->nz, g->st, g->stream));
  BicgState s;
  PF_TRY((run_bicgstab<double, UNI>(g, V, x, false, b, g->r64, g->p64, g->v64, g->rt64, g->t64, g->st, &s)));
  BicgState tr;
  PF_TRY(true_residual<UNI>(g, V, x, nullptr, b, o.tol, o.norm, &tr));
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
pf_status solve_mixed(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, pf_report* rep) {
  const OpView<double> V = view64(g, op);
  const OpView<float> W = view32(g, op);
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_impose(x, b, V.dinv, g->N, g->stream));
  int iters = 0, ref = 0, status = PF_E_NOCONV;
  BicgState tr{};
  bool have_d = false;
  for (;;) {
    PF_TRY(true_residual<UNI>(g, V, x, have_d ? g->d32 : nullptr, b, o.tol, o.norm, &tr));
    if (tr.done) {
      status = PF_OK;
      break;
    }
    if (ref >= o.max_refine || iters >= o.max_iter) {
      status = PF_E_NOCONV;
      break;
    }
    // FP32 inner solve A d = r (r = b - A x in b32), d0 = 0, to relative tolerance inner_tol; an inner
    // solve that stagnates is cut off after INNER_CAP iterations and its correction is kept
    PF_CK(cudaMemsetAsync(g->d32, 0, g->N * sizeof(float), g->stream));
    const int cap = o.max_iter - iters < INNER_CAP ? o.max_iter - iters : INNER_CAP;
    PF_TRY(set_state(g, g->st2, o.inner_tol, PF_NORM_REL2, cap));
    BicgState s;
    PF_TRY((run_bicgstab<float, UNI>(g, W, g->d32, true, g->b32, g->r32, g->p32, g->v32, g->rt32, g->t32, g->st2,
                                     &s)));
    iters += s.iter;
    have_d = true;
    ++ref;
    if (trace_level() > 0)
      fprintf(stderr, "[pf] mixed op %d refinement %d: true residual %.3e, inner status %d iters %d\n", op, ref,
              measure_of(tr, o.norm), s.status, s.iter);
    if (s.status == PF_E_BREAKDOWN && s.iter == 0) {
      status = PF_E_BREAKDOWN;
      break;
    }
    if (!isfinite(tr.rnorm2)) {
      status = PF_E_BREAKDOWN;
      break;
    }
  }
  rep->status = status;
  rep->iterations = iters;
  rep->refinements = ref;
  rep->residual = measure_of(tr, o.norm);
  return PF_OK;
}

pf_status solve_dev(pf_grid* g, int op, const double* b, double* x, const pf_solve_opts& o, pf_report* rep) {
  const bool uni = op == PF_OP_PF1;
  if (o.precision == PF_MIXED)
    return uni ? solve_mixed<true>(g, op, b, x, o, rep) : solve_mixed<false>(g, op, b, x, o, rep);
  return uni ? solve_fp64<true>(g, op, b, x, o, rep) : solve_fp64<false>(g, op, b, x, o, rep);
}

pf_status check_opts(const pf_solve_opts& o) {
  if (o.max_iter < 1 || !(o.tol > 0) || (o.norm != PF_NORM_REL2 && o.norm != PF_NORM_ABSINF) ||
      (o.precision != PF_FP64 && o.precision != PF_MIXED) || !(o.inner_tol > 0 && o.inner_tol < 1) ||
      o.max_refine < 1)
    return fail(PF_E_INVAL, "invalid pf_solve_opts");
  return PF_OK;
}

pf_status update_pf2(pf_grid* g) {
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_eps_diag(g->dsum, g->sig, g->solvent, g->nx, g->ny, g->nz, g->diag2,
                                                  g->dinv2, g->dinv2_32, g->stream));
  return PF_OK;
}

// Step a1 on the device from the stored eps, solvent mask and charges: harmonic faces (Eqs. 15-18
// with zero jump) in FP64 and FP32, diagonals and Jacobi scalings of the three operators, the
// trilinear fixed-charge source (Eq. 3).  kappa (PF2) is reset to zero.  Sets g->err when a charge
// lies outside the grid.
pf_status build_operators(pf_grid* g) {
  const long N = g->N;
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_faces(g->eps, g->nx, g->ny, g->nz, g->h, g->wE, g->wN, g->wU, g->dsum,
                                               g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wE, g->wE32, N, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wN, g->wN32, N, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_to_f32(g->wU, g->wU32, N, g->stream));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_eps_diag(g->dsum, nullptr, nullptr, g->nx, g->ny, g->nz, g->diagP, g->dinvP,
                                                  g->dinvP32, g->stream));
  PF_CK(cudaMemsetAsync(g->sig, 0, N * sizeof(double), g->stream));
  PF_TRY(update_pf2(g));
  const double wc = g->eps_s * g->lc * g->lc / (g->h * g->h);
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_pf1_dinv(g->solvent, g->nx, g->ny, g->nz, 1.0 / (6.0 * wc + g->eps_s),
                                                  g->dinv1, g->dinv1_32, g->stream));
  PF_CK(cudaMemsetAsync(g->ffix, 0, N * sizeof(double), g->stream));
  PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), g->stream));
  if (g->nq > 0)
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_spread(g->dch, g->nq, g->origin[0], g->origin[1], g->origin[2], g->h,
                                                  g->lam, g->nx, g->ny, g->nz, g->ffix, g->err, g->stream));
  return PF_OK;
}

}  // namespace

// Device bytes that pf_create_grid allocates for n_nodes nodes (used for the serving budget).
size_t pf_internal_grid_bytes(long n_nodes) {
  const size_t per_node = 30 * sizeof(double) + pf::MAXSP * sizeof(double) + 16 * sizeof(float) + 1;
  return (size_t)n_nodes * per_node + (size_t)pf::max_partial_blocks() * pf::NPART * sizeof(double) + 4096;
}

extern "C" {

void pf_default_solve_opts(pf_solve_opts* o) {
  if (!o) return;
  o->max_iter = 20000;
  o->tol = 1e-10;
  o->norm = PF_NORM_REL2;
  o->precision = PF_FP64;
  o->inner_tol = 0.1;
  o->max_refine = 64;
}

void pf_default_nl_opts(pf_nl_opts* o) {
  if (!o) return;
  o->omega = 0.3;
  o->tol_outer = 1e-9;
  o->max_outer = 500;
  pf_default_solve_opts(&o->lin);
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
  g->h = h_A;
  for (int a = 0; a < 3; ++a) g->origin[a] = origin_A[a];
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  pf_status s = allocate(g);
  if (s != PF_OK) {
    free_all(g);
    delete g;
    return s;
  }
  g->L = pf::make_launch(nx, ny, nz, g->stream);
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
  for (long i = 0; i < g->N; ++i)
    if (!(c->eps[i] > 0) || c->solvent[i] > 1) return fail(PF_E_INVAL, "eps must be > 0 and solvent 0/1");
  // species constants of Eq. (1): v_i = 4 pi a^3/3, v0 = mean volume, p_i = v_i/v0, Gamma^B = 1 - sum v cB
  const double molar = NAVO * 1e-27;
  double v[PF_MAX_SPECIES], v0 = 0.0, gB = 1.0, q = 0.0, qs = 0.0;
  const int ns = c->n_species;
  for (int i = 0; i < ns; ++i) {
    const pf_species& s = c->species[i];
    if (!(s.radius_A > 0) || !(s.bulk_M >= 0)) return fail(PF_E_INVAL, "species need radius > 0 and bulk >= 0");
    v[i] = 4.0 * M_PI * s.radius_A * s.radius_A * s.radius_A / 3.0;
    v0 += v[i];
  }
  v0 /= ns;
  pf::SpeciesParams sp{};
  sp.ns = ns;
  for (int i = 0; i < ns; ++i) {
    const pf_species& s = c->species[i];
    const double cB = s.bulk_M * molar;
    sp.z[i] = s.z;
    sp.p[i] = v[i] / v0;
    sp.lvc[i] = cB > 0 ? log(v[i] * cB) : -INFINITY;
    sp.lcB[i] = cB > 0 ? log(cB) : -INFINITY;
    gB -= v[i] * cB;
    q += s.z * cB;
    qs += fabs((double)s.z) * cB;
  }
  if (!(gB > 0)) return fail(PF_E_INVAL, "bulk void fraction Gamma^B <= 0");
  if (fabs(q) > 1e-12 * (qs > 0 ? qs : 1.0)) return fail(PF_E_INVAL, "bath is not electroneutral");
  sp.lgB = log(gB);
  g->T = c->T_K;
  g->Tv = KB * g->T / QE;
  g->lam = QE * QE / (EPS0 * KB * g->T * 1e-10);
  sp.lam = g->lam;
  g->sp = sp;
  g->molar = molar;
  g->eps_s = c->eps_s;
  g->lc = c->lc_A;
  g->lo_hat = c->phi_zlo_V / g->Tv;
  g->hi_hat = c->phi_zhi_V / g->Tv;

  const long N = g->N;
  PF_CK(cudaMemcpyAsync(g->eps, c->eps, N * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  PF_CK(cudaMemcpyAsync(g->solvent, c->solvent, N, cudaMemcpyHostToDevice, g->stream));
  if (g->dch) {
    cudaFree(g->dch);
    g->dch = nullptr;
  }
  g->nq = c->n_charges;
  if (g->nq > 0) {
    PF_CK(cudaMalloc(&g->dch, sizeof(double) * 4 * g->nq));
    PF_CK(cudaMemcpyAsync(g->dch, c->charges, sizeof(double) * 4 * g->nq, cudaMemcpyHostToDevice, g->stream));
  }
  PF_TRY(build_operators(g));
  PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  PF_CK(cudaStreamSynchronize(g->stream));
  if (*g->host_err) return fail(PF_E_INVAL, "a fixed charge lies outside the grid");
  g->have_coeffs = true;
  return PF_OK;
}

pf_status pf_set_kappa(pf_grid* g, const double* kappa, int mem) {
  if (!g || !kappa) return fail(PF_E_INVAL, "grid and kappa are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  PF_CK(cudaMemcpyAsync(g->sig, kappa, g->N * sizeof(double),
                        mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
  PF_TRY(update_pf2(g));
  PF_CK(cudaStreamSynchronize(g->stream));
  return PF_OK;
}

pf_status pf_linear_solve(pf_grid* g, int op, const double* b, double* x, int mem, const pf_solve_opts* opts,
                          pf_report* report) {
  if (!g || !b || !x) return fail(PF_E_INVAL, "grid, b and x are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  if (op != PF_OP_POISSON && op != PF_OP_PF1 && op != PF_OP_PF2) return fail(PF_E_INVAL, "unknown operator");
  if (mem != PF_MEM_HOST && mem != PF_MEM_DEVICE) return fail(PF_E_INVAL, "mem must be PF_MEM_HOST or PF_MEM_DEVICE");
  pf_solve_opts o;
  if (opts) o = *opts; else pf_default_solve_opts(&o);
  PF_TRY(check_opts(o));
  pf_report rep{};
  const size_t bytes = g->N * sizeof(double);
  PF_CK(cudaEventRecord(g->ev0, g->stream));
  const double* bd = b;
  double* xd = x;
  if (mem == PF_MEM_HOST) {
    PF_CK(cudaMemcpyAsync(g->bb, b, bytes, cudaMemcpyHostToDevice, g->stream));
    PF_CK(cudaMemcpyAsync(g->xb, x, bytes, cudaMemcpyHostToDevice, g->stream));
    bd = g->bb;
    xd = g->xb;
  }
  PF_TRY(solve_dev(g, op, bd, xd, o, &rep));
  if (mem == PF_MEM_HOST) PF_CK(cudaMemcpyAsync(x, g->xb, bytes, cudaMemcpyDeviceToHost, g->stream));
  PF_CK(cudaEventRecord(g->ev1, g->stream));
  PF_CK(cudaEventSynchronize(g->ev1));
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
  prof_resolve(g);
  rep.time_ms = ms;
  if (report) *report = rep;
  if (rep.status != PF_OK)
    return fail((pf_status)rep.status, rep.status == PF_E_NOCONV ? "linear solve did not converge"
                                                                  : "BiCGSTAB breakdown");
  return PF_OK;
}

pf_status pf_nonlinear_solve(pf_grid* g, const pf_nl_opts* opts, pf_result* res) {
  if (!g || !res) return fail(PF_E_INVAL, "grid and result are required");
  if (!g->have_coeffs) return fail(PF_E_INVAL, "pf_set_coeffs must come first");
  pf_nl_opts o;
  if (opts) o = *opts; else pf_default_nl_opts(&o);
  PF_TRY(check_opts(o.lin));
  if (!(o.omega >= 0 && o.omega < 1) || !(o.tol_outer > 0) || o.max_outer < 1)
    return fail(PF_E_INVAL, "invalid pf_nl_opts");
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const long N = g->N;
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
  // Table 4 step 4: PF2 with rho' = Psi = 0 -> Phi_0
  PF_CK(cudaMemsetAsync(g->phi0, 0, N * sizeof(double), s));
  PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_set_dirichlet(g->phi0, g->lo_hat, g->hi_hat, nx, ny, nz, s));
  PF_CK(cudaMemsetAsync(g->psi, 0, N * sizeof(double), s));
  PF_LAUNCH(g, PF_PROF_OTHER,
            pf::launch_pf2_rhs(g->psi, g->solvent, g->ffix, g->eps_s, g->lo_hat, g->hi_hat, nx, ny, nz, g->b2, s));
  PF_TRY(solve_dev(g, PF_OP_POISSON, g->b2, g->phi0, o.lin, &rep));
  res->lin_iters_first = rep.iterations;
  res->lin_iters_total += rep.iterations;
  if (rep.status != PF_OK) st = (pf_status)rep.status;
  for (int outer = 1; st == PF_OK && outer <= o.max_outer; ++outer) {
    // Eq. (1) at Phi_0 -> b_PF1 = -lambda rho, kappa, PF2 right-hand-side part (Table 4 steps 5-6)
    PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, nx, ny, nz, g->b1, g->sig,
                                                 g->c2, nullptr, nullptr, nullptr, g->err, s));
    PF_TRY(update_pf2(g));
    PF_TRY(solve_dev(g, PF_OP_PF1, g->b1, g->psi, o.lin, &rep));  // Eq. (12)
    res->lin_iters_total += rep.iterations;
    if (rep.status != PF_OK) { st = (pf_status)rep.status; break; }
    PF_LAUNCH(g, PF_PROF_OTHER,
              pf::launch_pf2_rhs(g->psi, g->solvent, g->c2, g->eps_s, g->lo_hat, g->hi_hat, nx, ny, nz, g->b2, s));
    PF_CK(cudaMemcpyAsync(g->phi, g->phi0, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PF_TRY(solve_dev(g, PF_OP_PF2, g->b2, g->phi, o.lin, &rep));  // Eq. (13)
    res->lin_iters_total += rep.iterations;
    if (rep.status != PF_OK) { st = (pf_status)rep.status; break; }
    // Table 4 step 7: relax and test
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_relax(g->phi0, g->phi, o.omega, N, g->part, g->ticket, g->delta, s));
    PF_CK(cudaMemcpyAsync(g->host_delta, g->delta, sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CK(cudaStreamSynchronize(s));
    if (*g->host_err) { st = PF_E_GAMMA; break; }
    res->outer_iters = outer;
    res->delta = *g->host_delta;
    if (trace_level() > 0) fprintf(stderr, "[pf] outer %d delta %.6e lin_total %d\n", outer, res->delta, res->lin_iters_total);
    if (res->delta <= o.tol_outer) break;
    if (outer == o.max_outer) st = PF_E_NOCONV;
  }
  // outputs at the final potential
  PF_CK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
  PF_LAUNCH(g, PF_PROF_FERMI, pf::launch_fermi(g->phi0, g->solvent, g->ffix, g->sp, nx, ny, nz, nullptr, nullptr,
                                               nullptr, g->Cbuf, g->Sbuf, g->Gbuf, g->err, s));
  const cudaMemcpyKind kind = res->mem == PF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (res->phi_V) {
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->phi0, g->Tv, g->phi, N, s));
    PF_CK(cudaMemcpyAsync(res->phi_V, g->phi, N * sizeof(double), kind, s));
  }
  if (res->C_M) {
    const long nc = N * g->sp.ns;
    PF_LAUNCH(g, PF_PROF_OTHER, pf::launch_scale(g->Cbuf, 1.0 / g->molar, g->Cbuf, nc, s));
    PF_CK(cudaMemcpyAsync(res->C_M, g->Cbuf, nc * sizeof(double), kind, s));
  }
  if (res->S) PF_CK(cudaMemcpyAsync(res->S, g->Sbuf, N * sizeof(double), kind, s));
  if (res->Gamma) PF_CK(cudaMemcpyAsync(res->Gamma, g->Gbuf, N * sizeof(double), kind, s));
  if (res->Psi) PF_CK(cudaMemcpyAsync(res->Psi, g->psi, N * sizeof(double), kind, s));
  PF_CK(cudaMemcpyAsync(g->host_err, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PF_CK(cudaEventRecord(g->ev1, s));
  PF_CK(cudaEventSynchronize(g->ev1));
  if (*g->host_err && st == PF_OK) st = PF_E_GAMMA;
  float ms = 0.f;
  PF_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
  prof_resolve(g);
  res->time_ms = ms;
  res->status = st;
  if (st != PF_OK) return fail(st, "nonlinear solve ended with status " + std::to_string((int)st));
  return PF_OK;
}

}  // extern "C"
