// pf_internal.cuh -- types and kernel launchers shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pf_gb300.h"

namespace pf {

constexpr int TX = 32;           // tile width in x (one warp per row)
constexpr int TY = 8;            // tile height in y
constexpr int NTHREADS = TX * TY;
constexpr int ZC = 32;           // interior planes per z-chunk of a tile (default; Geom::zc may choose another)
constexpr int MAXSP = 8;
constexpr int NPART = 16;        // per-block partial values reduced by the last block
constexpr int HBX = TX + 8;      // TMA halo box: x from x0-4 (16-byte aligned start) to x0+TX+3
constexpr int HBY = TY + 2;      // halo box rows y0-1 .. y0+TY

// Tiles in x and y.  With edges on, a grid whose extent in x (y) is one more than a multiple of TX (TY) -- every
// 2^k + 1 grid -- gets no tile for its last column (row): the tile next to it computes those nodes in its halo
// slots (edge nodes), so no block spends a whole tile on a single column or row.  That pays when a launch has
// several tiles per block; a grid with fewer tiles than the GPU holds at once keeps the narrow tiles, which run
// beside the others.
__host__ __device__ inline bool edge_x(int nx, int edges) { return edges && nx > TX && nx % TX == 1; }
__host__ __device__ inline bool edge_y(int ny, int edges) { return edges && ny > TY && ny % TY == 1; }
__host__ __device__ inline int tiles_x(int nx, int edges) { return edge_x(nx, edges) ? nx / TX : (nx + TX - 1) / TX; }
__host__ __device__ inline int tiles_y(int ny, int edges) { return edge_y(ny, edges) ? ny / TY : (ny + TY - 1) / TY; }

// Device arrays use a padded layout: node (i,j,k) at i + px*j + px*ny*k with px a multiple of 8,
// so every row starts on a 32-byte boundary and rows are valid TMA strides.
struct Geom {
  int nx, ny, nz, px;
  long plane;  // px * ny
  long np;     // plane * nz (allocated elements)
  long n;      // nx * ny * nz (nodes)
  int zc;      // interior z-planes per tile of the stencil kernels
  int edges;   // 1: the last column / row of a 2^k + 1 grid are edge nodes of the tiles next to them
};

inline Geom make_geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.px = (nx + 7) / 8 * 8;
  g.plane = (long)g.px * ny;
  g.np = g.plane * nz;
  g.n = (long)nx * ny * nz;
  g.zc = ZC;
  g.edges = 0;
  return g;
}

// Device-resident BiCGSTAB scalars (Table 3); written only by the last block of a kernel.
struct BicgState {
  double rho;      // r~ . r of the current residual
  double alpha, omega, beta;
  double bnorm2;   // ||b||_2^2 of the system
  double rnorm2, rinf;   // ||r||_2^2, ||r||_inf of the latest residual
  double snorm2, sinf;
  double tol;      // tolerance as given
  double tol2;     // REL2: max(tol^2 ||b||^2, tol_r0^2 ||r0||^2)
  double tol_r0;   // additional tolerance relative to the first residual of the solve (0: none)
  double r0norm2;  // ||r0||_2^2 of the first residual computed since the state was reset (< 0: none yet)
  int norm;        // 0 REL2, 1 ABSINF
  int iter, max_iter;
  int done, status, sexit;
  unsigned int ticket;   // arrival counter of the last-block reduction
  int pad;
};

// Tensor maps of one stencil kernel: NH arrays read at neighbours, loaded as halo boxes (HBX x HBY at (x0-4, y0-1,
// k)), and NC arrays read at the node only, loaded as row boxes (HBX x TY at (x0-4, y0, k): the halo box without
// its first and last row) -- or as halo boxes when the grid has edge nodes (Geom::edges), which lie in those rows.
template <int NH, int NC>
struct Maps {
  CUtensorMap h[NH];
  CUtensorMap c[NC > 0 ? NC : 1];
};

// Slots of the stencil kernels (the API fills the maps in this order):
//   phase B:   halo {r, v, dinv, wE, wN},       centre {r~, wU}     (variable-face operators)
//              halo {r, v, dinv},               centre {r~}         (PF1)
//   phase C+A: halo {r, v, t, p, dinv, wE, wN}, centre {x, r~, wU}  (FP64 variable-face operators)
//              halo {r, v, t, p, dinv, gh},     centre {x, r~}      (FP32 variable-face operators)
//              halo {r, v, t, p, dinv},         centre {x, r~}      (PF1)
//   residual:  halo {x, dinv, wE, wN} (PF1: {x, dinv}),             centre {b, diag, wU} (PF1: {b})
// gh = h^2 / (2 eps) per node: the FP32 phase C+A kernel, bound by DRAM traffic, forms each harmonic face
// (Eqs. 15-18 with zero jump) as 1 / (gh_a + gh_b) = 2 eps_a eps_b / ((eps_a + eps_b) h^2) instead of reading
// three face arrays; the FP32 phase B kernel, bound by instruction issue, reads the stored FP32 faces.
template <typename T> constexpr bool ca_face_from_gh() { return sizeof(T) == 4; }
template <typename T, bool UNI> struct SlotsB { static constexpr int NH = UNI ? 3 : 5, NC = UNI ? 1 : 2; };
template <typename T, bool UNI> struct SlotsCA {
  static constexpr int NH = UNI ? 5 : (ca_face_from_gh<T>() ? 6 : 7), NC = UNI ? 2 : (ca_face_from_gh<T>() ? 2 : 3);
};
template <bool UNI> struct SlotsRes { static constexpr int NH = UNI ? 2 : 4, NC = UNI ? 1 : 3; };
//   CG pass:   halo {r, w, s, dinv, wE, wN}, centre {p, x, wU}  (FP64 variable-face operators)
//              halo {r, w, s, dinv, gh},     centre {p, x}      (FP32 variable-face operators)
//              halo {r, w, s, dinv},         centre {p, x}      (PF1)
template <typename T, bool UNI> struct SlotsCG {
  static constexpr int NH = UNI ? 4 : (ca_face_from_gh<T>() ? 5 : 6), NC = UNI ? 2 : (ca_face_from_gh<T>() ? 2 : 3);
};

struct Launch {
  int ntiles;
  cudaStream_t stream;
  unsigned long long wait_limit;  // clock cycles a block may wait on one TMA stage
};

// species constants of Eq. (1) in scaled units
struct SpeciesParams {
  int ns;
  double z[MAXSP];
  double lvc[MAXSP];    // ln(v_i cB_i) (or -inf when cB_i = 0)
  double p[MAXSP];      // v_i / v0
  double lcB[MAXSP];    // ln cB_i
  double inv_v[MAXSP];  // 1 / v_i, v_i = 4 pi a_i^3 / 3
  double inv_p[MAXSP];  // 1 / p_i
  double lgB;           // ln Gamma^B
  double lnn;           // ln(1 + number of species with cB_i > 0)
  double lam;           // lambda
};

// The same constants as double-float pairs (value = hi + lo) for the FP32-pipe form of the pointwise step.
struct SpeciesDF {
  int ns;
  int present[MAXSP];                   // cB_i > 0
  float z[MAXSP];
  float phi[MAXSP], plo[MAXSP];         // p_i
  float inv_p[MAXSP];                   // 1 / p_i (bracket only)
  float chi[MAXSP], clo[MAXSP];         // ln(v_i cB_i) - p_i ln Gamma^B
  float ivhi[MAXSP], ivlo[MAXSP];       // 1 / v_i
  float lnn;                            // ln(1 + number of species present)
  float lgB;                            // ln Gamma^B (the cold start)
  float lamhi, lamlo;                   // lambda
};
SpeciesDF species_df(const SpeciesParams& sp);

// host: species constants of Eq. (1) from a caller's species list (nullptr, or why the list is invalid);
// tv = k_B T / e in volts, molar = the mol/L -> A^-3 factor
const char* species_params(int ns, const pf_species* species, double T_K, SpeciesParams* out, double* tv,
                           double* molar);

int tiles_for(int nx, int ny, int nz, int zc = ZC, int edges = 0);
// edges for a single grid: on when its stencil launches hold several tiles per block
int edges_for(int nx, int ny, int nz);
int max_partial_blocks();

// host: encode a 3D tensor map over a padded device array (halo box when halo, else centre box)
// box: BOX_HALO (HBX x HBY) or BOX_ROWS (HBX x TY)
enum { BOX_HALO = 1, BOX_ROWS = 2 };
bool encode_map(CUtensorMap* m, const void* base, const Geom& g, int elem_bytes, int box);

// ---- setup (a1) ----
// FP64 faces and their sum per node, and gh = h^2 / (2 eps) in FP32 for the FP32 phase C+A kernel
cudaError_t launch_faces(const double* eps, const Geom& g, double h, double* wE, double* wN, double* wU,
                         double* dsum, float* gh32, cudaStream_t s);
cudaError_t launch_spread(const double* charges, int nq, double ox, double oy, double oz, double h, double lam,
                          const Geom& g, double* f, int* err, cudaStream_t s);
cudaError_t launch_eps_diag(const double* dsum, const double* sig, const uint8_t* smask, const Geom& g, double* diag,
                            double* dinv, float* dinv32, cudaStream_t s);
cudaError_t launch_pf1_dinv(const uint8_t* solvent, const Geom& g, double dinvc, double* dinv, float* dinv32,
                            cudaStream_t s);
cudaError_t launch_to_f32(const double* a, float* b, long n, cudaStream_t s);
cudaError_t launch_impose(double* x, const double* b, const double* dinv, long n, cudaStream_t s);
// compact (x fastest, pitch nx) <-> padded (pitch px) copies of `count` consecutive fields;
// type 0 double, 1 uint8
cudaError_t launch_pack(const void* src, void* dst, const Geom& g, int type, cudaStream_t s);
cudaError_t launch_unpack(const double* src, double* dst, const Geom& g, int count, cudaStream_t s);

// ---- BiCGSTAB (Table 3) ----
// keep_r0 != 0 keeps r0norm2 and bnorm2 of the previous state (later refinement steps of one solve)
cudaError_t launch_set_state(BicgState* st, double tol, int norm, int max_iter, double tol_r0, int keep_r0,
                             cudaStream_t s);
// b.b over the two Dirichlet planes -> st->bnorm2 (uses the partials buffer and the state's ticket)
cudaError_t launch_plane_bb(const double* b, const Geom& g, double* part, BicgState* st, cudaStream_t s);
// st->done = 1 (the stencil kernels then skip the state's grid)
cudaError_t launch_mark_done(BicgState* st, cudaStream_t s);
// *status = 7 when a bounded wait on a barrier that never completes gives up after `limit` cycles, else 0
cudaError_t launch_wait_probe(unsigned long long limit, int* status, cudaStream_t s);
// r = r~ = b, p = v = t = 0 on interior nodes (x0 = 0); partials b.b, r.r, max|r|
template <typename T>
cudaError_t launch_init_zero(const T* b, const Geom& g, T* r, T* rt, T* p, T* v, T* t, double* part, BicgState* st,
                             cudaStream_t s);
// Options of the FP64 residual: need_bb = 0 reuses b.b kept in the state (a later refinement step of the same
// right-hand side); need_max = 0 skips max |r| (2-norm stop test); st2 != nullptr starts the FP32 inner solve
// of refinement in the same pass: r = r~ = (float) r, p = v = t = d = 0 and st2 from ||r||^2.
struct ResidualExtras {
  int need_bb = 1, need_max = 1;
  float *r = nullptr, *rt = nullptr, *p = nullptr, *v = nullptr, *t = nullptr, *d = nullptr;
  BicgState* st2 = nullptr;
};
// r = b - A x (x holds b on identity rows) in FP64; init = 1 also writes r~ = r, p = v = t = 0 and starts
// the BiCGSTAB state; init = 0 writes r32 = (float) r (or starts the inner solve, see ResidualExtras) and the
// refinement state
template <bool UNI>
cudaError_t launch_residual(const Maps<SlotsRes<UNI>::NH, SlotsRes<UNI>::NC>& m, const Geom& g, double wc,
                            double diagc, int init, double* r, double* rt, double* p, double* v, double* t, float* r32,
                            double* part, BicgState* st, const Launch& L, const ResidualExtras& ex = ResidualExtras());
template <typename T, bool UNI>
cudaError_t launch_phase_b(const Maps<SlotsB<T, UNI>::NH, SlotsB<T, UNI>::NC>& m, const Geom& g, T wc, T* t, double* part,
                           BicgState* st, const Launch& L);
template <typename T, bool UNI>
cudaError_t launch_phase_ca(const Maps<SlotsCA<T, UNI>::NH, SlotsCA<T, UNI>::NC>& m, const Geom& g, T wc, T* x, T* r_out,
                            T* p_out, T* v_out, double* part, BicgState* st, int prime, const Launch& L);
// One pass of Jacobi-preconditioned CG (Chronopoulos-Gear form, OpCG): prime = 1 is the start pass.
template <typename T, bool UNI>
cudaError_t launch_cg_pass(const Maps<SlotsCG<T, UNI>::NH, SlotsCG<T, UNI>::NC>& m, const Geom& g, T wc, T* r_out,
                           T* w_out, T* s_out, T* p, T* x, double* part, BicgState* st, int prime, const Launch& L);
cudaError_t launch_add_f32(double* x, const float* d, long n, cudaStream_t s);

// ---- nonlinear step (Eq. 1, Eq. 11-13, Table 4) ----
// ulast: per-node ln Gamma of the previous call, read when warm != 0 (Newton start) and rewritten; with
// u32start != nullptr a warm start reads that FP32 copy instead (the one the double-float step keeps)
cudaError_t launch_fermi(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesParams& sp,
                         const Geom& g, double* b1, double* sig, double* c2, double* C, double* S, double* G,
                         double* ulast, int warm, int* err, cudaStream_t s, const float* u32start = nullptr);
// The in-loop pointwise step of the mixed-precision solve in double-float arithmetic on the FP32 pipes:
// b1 = -lambda rho, kappa and kappa phi0 + ffix as the FP64 step writes them (rho to about 1e-14 relative,
// kappa, which only steers the iteration, to FP32); u32 holds each node's ln Gamma (warm start, rewritten).
cudaError_t launch_fermi_df(const double* phi0, const uint8_t* solvent, const double* ffix, const SpeciesDF& sp,
                            const Geom& g, double* b1, double* sig, double* c2, float* u32, int warm, int* err,
                            cudaStream_t s);
cudaError_t launch_pf2_rhs(const double* psi, const uint8_t* solvent, const double* c2, double eps_s, double lo,
                           double hi, const Geom& g, double* b2, cudaStream_t s);
cudaError_t launch_relax(double* phi0, const double* phi, double omega, long n, double* part, unsigned int* ticket,
                         double* delta, cudaStream_t s);
cudaError_t launch_scale(const double* a, double s, double* out, long n, cudaStream_t st);

// ---- Anderson acceleration of the outer iteration (history of at most AA_MAX columns) ----
constexpr int AA_MAX = 8;
struct AAPtrs {
  const double* dF[AA_MAX];
  const double* dX[AA_MAX];
};
struct AACoef {
  double g[AA_MAX];
};
cudaError_t launch_aa_residual(const double* gval, const double* x, double* f, double* fprev, double* xprev,
                               double* dF, double* dX, int have_prev, long n, double* part, unsigned int* ticket,
                               double* fmax, cudaStream_t s);
// out[j] = dF_new . dF_j, out[AA_MAX + j] = dF_j . f for j < k
cudaError_t launch_aa_dots(const AAPtrs& cols, int k, const double* dFnew, const double* f, long n, double* part,
                           unsigned int* ticket, double* out, cudaStream_t s);
cudaError_t launch_aa_update(const AAPtrs& cols, const AACoef& gam, int k, double beta, double* x, const double* f,
                             long n, cudaStream_t s);
cudaError_t launch_set_dirichlet(double* x, double lo, double hi, const Geom& g, cudaStream_t s);

}  // namespace pf
