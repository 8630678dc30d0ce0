// pf_grid.cuh -- the library's per-grid state (struct pf_grid) and the host helpers that the single-grid
// solver (pf_api.cu) and the batched solver (pf_batch.cu) share: error reporting, stream-ordered device
// allocation, launch profiling, TMA descriptor cache, operator and Krylov array views.
#pragma once
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

#include <nvtx3/nvToolsExt.h>

#include "../../include/pf_gb300.h"
#include "pf_internal.cuh"

namespace pfi {

using pf::BicgState;

pf_status fail(pf_status s, const std::string& msg);
pf_status cuda_fail(cudaError_t e, const char* what);

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

constexpr int CHUNK = 8;         // BiCGSTAB iterations launched between two host checks of the done flag
constexpr int INNER_CAP = 1000;  // FP32 iterations per refinement step at most
// An FP32 inner solve that can end the refinement (its start ||r|| within 1/inner_tol of the solve's target T)
// stops at FINAL_INNER_MARGIN * T instead of inner_tol ||r||: the next FP64 true residual decides
constexpr double FINAL_INNER_MARGIN = 0.5;
constexpr int PROF_SLOTS = 64;   // timed launches between two resolutions of the profiling events
constexpr unsigned long long WAIT_LIMIT = 4000000000ull;  // clock cycles (about 2 s) per TMA stage wait

}  // namespace pfi

struct pf_grid {
  int nx = 0, ny = 0, nz = 0;
  long N = 0;   // nodes
  pf::Geom geom{};
  double h = 1.0, origin[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  pf::Launch L{};
  bool have_coeffs = false;
  bool have_phi0 = false;    // phi0 holds a potential to warm-start from (last solve or pf_set_potential)
  bool ulast_valid = false;  // ulast holds the per-node ln Gamma of the last Fermi step on this problem
  bool u32_valid = false;    // ulast32 holds the FP32 ln Gamma of the last double-float Fermi step
  bool filter_on = false;    // a filter region (pf_set_filter) holds fixed potentials
  int charge_mode = 0;       // 0: charges spread (Eq. 3); 1: decomposition (Eqs. 5-10, pf_set_charge_mode)
  double eps_m = 0.0;        // the membrane dielectric when it is uniform (pf_set_coeffs), else NaN
  double *Gdec = nullptr, *bif = nullptr;  // G = phi* + phi^L and the interface right-hand side (mode 1)
  uint8_t* fmask = nullptr;  // its nodes (padded layout), allocated on first use
  double* fval = nullptr;    // their potentials in units of k_BT/e (padded layout)
  // problem constants
  double eps_s = 78.5, lc = 0.0, T = 298.15, Tv = 0.0, lam = 0.0, lo_hat = 0.0, hi_hat = 0.0, molar = 0.0;
  pf::SpeciesParams sp{};
  pf::SpeciesDF spd{};       // the same constants as double-float pairs
  // device arrays (padded layout)
  std::vector<void*> allocs;
  double *eps = nullptr, *wE = nullptr, *wN = nullptr, *wU = nullptr, *dsum = nullptr, *ffix = nullptr;
  uint8_t* solvent = nullptr;
  double *diagP = nullptr, *dinvP = nullptr, *diag2 = nullptr, *dinv2 = nullptr, *sig = nullptr, *dinv1 = nullptr;
  float *wE32 = nullptr, *wN32 = nullptr, *wU32 = nullptr;  // FP32 faces (phase B)
  float *gh32 = nullptr;  // h^2 / (2 eps): phase C+A's FP32 faces are 1 / (gh_a + gh_b)
  float *dinvP32 = nullptr, *dinv2_32 = nullptr, *dinv1_32 = nullptr;
  double *r64[2] = {nullptr, nullptr}, *p64[2] = {nullptr, nullptr}, *v64[2] = {nullptr, nullptr};
  double *rt64 = nullptr, *t64 = nullptr;
  float *r32[2] = {nullptr, nullptr}, *p32[2] = {nullptr, nullptr}, *v32[2] = {nullptr, nullptr};
  float *rt32 = nullptr, *t32 = nullptr, *d32 = nullptr, *b32 = nullptr, *ulast32 = nullptr;
  double *xb = nullptr, *bb = nullptr, *stage = nullptr;
  double *phi0 = nullptr, *phi = nullptr, *psi = nullptr, *b1 = nullptr, *c2 = nullptr, *b2 = nullptr;
  double *Cbuf = nullptr, *Sbuf = nullptr, *Gbuf = nullptr, *ulast = nullptr;
  double* part = nullptr;
  // Anderson acceleration of the outer loop (allocated on first use)
  int aa_alloc = 0;
  double *aa_f = nullptr, *aa_fprev = nullptr, *aa_xprev = nullptr, *aa_out = nullptr, *aa_host = nullptr;
  // the PF1 and PF2 solutions of the two outer iterations before the last one, newest first (pf_nl_opts.predict;
  // on first use; the pointers of a pair swap as the history moves on)
  double *xp_psi = nullptr, *xpp_psi = nullptr, *xp_phi = nullptr, *xpp_phi = nullptr;
  double *aa_dF[pf::AA_MAX] = {}, *aa_dX[pf::AA_MAX] = {};
  double* dch = nullptr;     // fixed charges (x, y, z, q) on the device
  int nq = 0;
  pf::BicgState* st = nullptr;   // FP64 solve / refinement state
  pf::BicgState* st2 = nullptr;  // FP32 inner solve state
  pf::BicgState* host_st = nullptr;  // pinned mirror
  int* err = nullptr;        // device error flag
  int* host_err = nullptr;   // pinned
  double* delta = nullptr;
  unsigned int* ticket = nullptr;
  double* host_delta = nullptr;
  void* hostblk = nullptr;   // pinned block holding host_st, host_err, host_delta and aa_host
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // TMA descriptors, keyed by (array, halo box?)
  std::map<std::pair<const void*, int>, CUtensorMap> maps;
  // profiling: event pairs around launches in two halves of PROF_SLOTS pairs; a half is read back when the other
  // fills up (its events long complete by then) or at the end of a solve, never at the solve's own host checks
  int prof_on = 0;
  long long launches = 0;
  long long pcount[PF_PROF_KINDS] = {};
  double pms[PF_PROF_KINDS] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<int> pkind;
  int np = 0;    // pairs recorded in the current half
  int half = 0;  // the current half
  int nold = 0;  // pairs of the other half not yet read back
};

namespace pfi {

int trace_level();

// NVTX range for profilers (a no-op unless a tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
void prof_resolve(pf_grid* g);
int prof_begin(pf_grid* g, int n_launches);
void prof_end(pf_grid* g, int slot, int kind);

#define PF_LAUNCH(g, kind, call)                  \
  do {                                            \
    const int slot_ = prof_begin((g), 1);         \
    PF_CK(call);                                  \
    prof_end((g), slot_, (kind));                 \
  } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the grid's stream), so creating and
// destroying grids does not synchronise the device while other grids run on other streams.
template <typename T>
pf_status dalloc(pf_grid* g, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 1;
  cudaError_t e = cudaMallocAsync(&q, bytes, g->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PF_E_OOM, std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                              cudaGetErrorString(e));
  }
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return PF_OK;
}

// ---- TMA descriptors ---------------------------------------------------------------------
template <typename T>
const CUtensorMap* tmap(pf_grid* g, const T* base, int box) {
  const auto key = std::make_pair(static_cast<const void*>(base), (int)sizeof(T) * 4 + box);
  auto it = g->maps.find(key);
  if (it != g->maps.end()) return &it->second;
  CUtensorMap m;
  if (!pf::encode_map(&m, base, g->geom, (int)sizeof(T), box)) return nullptr;
  return &(g->maps[key] = m);
}

template <int NH, int NC, typename T>
// centre_halo: the centre arrays as halo boxes, else as row boxes (-1: as the grid's own launches need them)
pf_status fill_maps(pf_grid* g, pf::Maps<NH, NC>* m, const T* const (&h)[NH], const T* const (&c)[NC],
                    int centre_halo = -1) {
  if (centre_halo < 0) centre_halo = g->geom.edges;
  for (int i = 0; i < NH; ++i) {
    const CUtensorMap* p = tmap(g, h[i], pf::BOX_HALO);
    if (!p) return fail(PF_E_CUDA, "cuTensorMapEncodeTiled failed");
    m->h[i] = *p;
  }
  for (int i = 0; i < NC; ++i) {
    const CUtensorMap* p = tmap(g, c[i], centre_halo ? pf::BOX_HALO : pf::BOX_ROWS);
    if (!p) return fail(PF_E_CUDA, "cuTensorMapEncodeTiled failed");
    m->c[i] = *p;
  }
  return PF_OK;
}

// The arrays of one operator in one precision: Jacobi scaling (0 on identity rows), FP64 diagonal,
// face arrays (null for the uniform PF1 operator), uniform face and diagonal, and for the FP32
// variable-face operators gh = h^2 / (2 eps) per node (phase C+A's faces).
template <typename T>
struct OpArrays {
  const T* dinv;
  const double* diag;
  const T *wE, *wN, *wU;
  double wc, diagc;
  const T* gh;
};

// Krylov vectors of one precision
template <typename T>
struct Krylov {
  T* r[2];
  T* p[2];
  T* v[2];
  T* rt;
  T* t;
};

double pf1_face(const pf_grid* g);
OpArrays<double> ops64(const pf_grid* g, int op);
OpArrays<float> ops32(const pf_grid* g, int op);
Krylov<double> kry64(pf_grid* g);
Krylov<float> kry32(pf_grid* g);
pf_status set_state(pf_grid* g, BicgState* dst, double tol, int norm, int max_iter, double tol_r0 = 0.0,
                    int keep_r0 = 0);
pf_status read_state(pf_grid* g, const BicgState* src, BicgState* out);
double measure_of(const BicgState& s, int norm);
pf_status check_opts(const pf_solve_opts& o);
pf_status update_pf2(pf_grid* g);
pf_status build_operators(pf_grid* g);
pf_status pack_in(pf_grid* g, const void* src, int mem, void* dst, int type);
pf_status unpack_out(pf_grid* g, const double* src, int count, double* dst, int mem);
pf_status ensure_aa(pf_grid* g, int m);
// The starting vector of a linear solve of the outer iteration (pf_nl_opts.predict) from the last solution x and
// the two before it (h0 newest; the pointers rotate): have = solutions so far (1: x only saved; 2: extrapolated
// with c_fallback; 3 and more: with c from the vector's own last two changes).  FP64 over the padded grid.
pf_status predict(pf_grid* g, double* x, double*& h0, double*& h1, int have, double c_fallback);
// the four FP64 vectors of pf_nl_opts.predict, allocated on first use
pf_status ensure_predict(pf_grid* g);
// Squared 2-norm stop of the FP32 inner solve of a refinement step, given the step's FP64 residual norm^2 rr and
// the solve's squared target t2 (REL2 only): FINAL_INNER_MARGIN^2 t2 when that is above inner_tol^2 rr, else 0
// (keep inner_tol)
double final_inner_tol2(const pf_solve_opts& o, double rr, double t2);
// st->tol2 = max(st->tol2, t2) on the device, in stream order
pf_status raise_tol2(pf_grid* g, BicgState* st, double t2, cudaStream_t s);
bool small_spd_solve(int k, const double (&A)[pf::AA_MAX][pf::AA_MAX], const double* b, double* x);

// The update at the end of an outer iteration (Table 4's relaxation, or Anderson acceleration of the same
// map when m > 0), split at its host read-backs so that a batch runs each stage over all of its grids
// between two synchronisations: stage 1 queues the update (relaxation) or f = Phi - Phi_0 with the history
// (Anderson) and the read-back of max |.| and the error flag; outer_delta gives delta once that landed;
// stage 2 queues the least-squares inner products (Anderson, when the iteration goes on and history
// exists; sets dots); stage 3 solves the small least-squares problem and updates Phi_0.
struct OuterUpdate {
  double Gm[pf::AA_MAX][pf::AA_MAX] = {};  // Gram matrix of the history columns, by ring slot
  int nact = 0, head = 0, kaa = 0, slot = 0;  // active columns, next slot, accelerated iterations, newest slot
  int act[pf::AA_MAX] = {};                // active slots, oldest first
  pf::AAPtrs cols{};
  bool dots = false;
};
// One problem of a batch (pf_batch.cu): its grid, where its outputs go, its options and its place in the
// per-problem state machine of the engine.
struct BatchMember {
  pf_grid* g = nullptr;
  pf_result* res = nullptr;
  pf_nl_opts o{};
  OuterUpdate U;
  double dprev = 1.0;   // delta of the previous outer iteration (forcing term)
  double dprev2 = 0.0;  // delta of the one before (pf_nl_opts.predict)
  double cpred = 0.0;   // extrapolation factor of this outer iteration's starting vectors
  int pred_have = 0;    // history length predict() is given in this outer iteration
  double inner_t2 = 0.0;  // squared stop of the next FP32 inner solve when it may end the refinement (else 0)
  int stage = 0;        // step of the nonlinear iteration (pf_batch.cu: Stage)
  int after = 0;        // stage to enter when the running linear solve ends
  // the linear solve in progress
  int op = 0, sub = 0, iters = 0, refs = 0;
  double eta = 0.0;     // forcing: also stop at eta ||r0||
  bool add_pending = false;
  bool fermi_warm = false;  // the first Fermi step may start Newton from the grid's last ln Gamma (warm start)
  pf_status st = PF_OK;
  long long tag = 0;    // the owner's handle
};

// The batched engine behind the server: problems join (engine_add, grid created on engine_stream) and
// leave (engine_step reports the tags of those that finished, their outputs written, and drops them)
// between steps; every step runs one outer iteration of all members in shared batched launches.
constexpr int ENGINE_TILES_PER_BLOCK = 4;
pf_status engine_create(int max_members, pf_batch** out);
cudaStream_t engine_stream(pf_batch* B);
pf_status engine_add(pf_batch* B, pf_grid* g, pf_result* res, const pf_nl_opts& o, long long tag);
pf_status engine_step(pf_batch* B, std::vector<long long>* finished);

pf_status outer_stage1(pf_grid* g, OuterUpdate& u, int m, double omega);
double outer_delta(const pf_grid* g, int m, double omega);
pf_status outer_stage2(pf_grid* g, OuterUpdate& u, int m, bool stop);
pf_status outer_stage3(pf_grid* g, OuterUpdate& u, int m, double omega, bool stop);

}  // namespace pfi
