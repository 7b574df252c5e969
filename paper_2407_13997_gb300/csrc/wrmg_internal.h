// Internal declarations shared by the translation units of libwrmg.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "wrmg.h"

#ifdef __CUDACC__
#define WR_HD __host__ __device__
#else
#define WR_HD
#endif

// Compile-time bounds: Navier-Stokes k <= 2 (Q3/Q2) and q <= 1 (DG(1)); the heat
// equation k <= 3 (Q3) and q <= 3 (DG(3)).
#define WR_MAX_NQ 5   // Gauss points per direction, k + 3
#define WR_MAX_NVL 4  // velocity nodes per cell and direction, k + 2
#define WR_MAX_NPL 3  // pressure nodes per cell and direction, k + 1
#define WR_MAX_NT 4   // temporal DoFs per slab, q + 1
#define WR_MAX_NTQ 5  // Gauss points in time for the forcing, q + 2

struct WrError : std::runtime_error {
  int code;
  WrError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// On failure the runtime's last-error slot is cleared as well, so that a failed call
// is reported once, here, and not again by a later launch check.
#define WR_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t wr_cuda_rc_ = (call);                                                   \
    if (wr_cuda_rc_ != cudaSuccess) {                                                   \
      cudaGetLastError();                                                               \
      throw WrError(wr_cuda_rc_ == cudaErrorMemoryAllocation ? WR_ERR_NOMEM : WR_ERR_CUDA, \
                    std::string(#call) + ": " + cudaGetErrorString(wr_cuda_rc_));       \
    }                                                                                   \
  } while (0)
// Description of the last failure of a call that takes no context (this thread's);
// wr_last_error(NULL) returns it.
void wr_set_context_free_error(const std::string& msg);
// Every kernel launch of the library is followed by WR_LAUNCH_CHECK, which also counts it.
void wr_count_launch();
void wr_count_launches(int64_t n);    // kernels of a replayed CUDA graph
void wr_uncount_launches(int64_t n);  // kernels captured into a graph, not launched
#define WR_LAUNCH_CHECK()        \
  do {                           \
    wr_count_launch();           \
    WR_CUDA(cudaGetLastError()); \
  } while (0)

// Reference-element tables (passed to kernels by value).  Reference interval
// [0, 1]; quadrature points xq with weights wq (Gauss-Legendre, k+3 points).
struct FeTables {
  double xq[WR_MAX_NQ], wq[WR_MAX_NQ];
  double Bv[WR_MAX_NQ][WR_MAX_NVL];  // velocity basis phi_i(xq)
  double Dv[WR_MAX_NQ][WR_MAX_NVL];  // phi_i'(xq)
  double Bp[WR_MAX_NQ][WR_MAX_NPL];  // pressure basis chi_i(xq)
  // 1D reference element matrices
  double m1[WR_MAX_NVL][WR_MAX_NVL];  // int phi_i phi_j
  double k1[WR_MAX_NVL][WR_MAX_NVL];  // int phi_i' phi_j'
  double d1[WR_MAX_NPL][WR_MAX_NVL];  // int chi_p phi_v'
  double c1[WR_MAX_NPL][WR_MAX_NVL];  // int chi_p phi_v
  double mp1[WR_MAX_NPL];             // int chi_p
  // DG(q) time matrices on the reference slab (see TimeMatrices in the docs)
  double Kt[WR_MAX_NT][WR_MAX_NT];     // int tau_a tau_b' + tau_a(0) tau_b(0)
  double Wt[WR_MAX_NT][WR_MAX_NT];     // int tau_a tau_b
  double tau0[WR_MAX_NT];              // tau_a(0)
  double T3[WR_MAX_NT][WR_MAX_NT][WR_MAX_NT];
  double tnode[WR_MAX_NT];             // right-Radau nodes
  double tq[WR_MAX_NTQ], wtq[WR_MAX_NTQ];
  double Tq[WR_MAX_NT][WR_MAX_NTQ];    // tau_a(tq_g)
  // 1D prolongation weights: fine node r (0..2p) of a coarse cell, coarse local node l
  double pv[2 * (WR_MAX_NVL - 1) + 1][WR_MAX_NVL];
  double pp[2 * (WR_MAX_NPL - 1) + 1][WR_MAX_NPL];
};

struct PhysParams {
  int kind, steady;
  double nu, conv, T;
  int n_modes;
  int mx[8], my[8];
  double amp[8];
  double t0 = 0.0;              // time at the start of slab 0
  const double* u0 = nullptr;   // slab-0 initial velocity: a spatial block (device), or null = exact u(t0)
};

struct LevelGeom {
  int n, k, q, N, nt, nv, np, S;
  int64_t ndofs;
  double h, dt;
  WR_HD int ncells() const { return n * n; }
  WR_HD int npatch() const { return (n + 1) * (n + 1); }
};

inline LevelGeom make_geom(int n, int k, int q, int N, double T) {
  LevelGeom g;
  g.n = n; g.k = k; g.q = q; g.N = N; g.nt = q + 1;
  g.nv = n * (k + 1) + 1;
  g.np = n * k + 1;
  g.S = 2 * g.nv * g.nv + g.np * g.np;
  g.ndofs = (int64_t)N * g.nt * g.S;
  g.h = 1.0 / n;
  g.dt = T / N;
  return g;
}

// Per-patch slot counts: velocity grid (2k+3)^2 per component, pressure (2k-1)^2.
inline int patch_nvg(int k) { return 2 * k + 3; }
inline int patch_npg(int k) { return 2 * k - 1; }
inline int patch_ms(int k) { return 2 * patch_nvg(k) * patch_nvg(k) + patch_npg(k) * patch_npg(k); }
// Elements of one stored ms x ms factor block, padded to a multiple of 16 bytes
// (the granule of the bulk copies that stream the blocks into shared memory).
inline int factor_elem_bytes(int precision) { return precision == WR_FP32 ? 4 : precision == WR_BF16 ? 2 : 8; }
inline int64_t block_elems(int ms, int precision) {
  const int64_t e = (int64_t)ms * ms;
  const int64_t g = precision == WR_FP32 ? 4 : precision == WR_BF16 ? 8 : 2;
  return (e + g - 1) / g * g;
}
inline int64_t factor_block_elems(int k, int precision) { return block_elems(patch_ms(k), precision); }
// Slot count per temporal DoF of the coarse block: the patch shape holds the
// 2x2 coarse mesh; the 3x3 coarse mesh of Q2/Q1 needs 2*5^2 + 4^2 = 66 slots.
inline int coarse_ms(int k, int n_coarse) { return n_coarse == 2 ? patch_ms(k) : 2 * 25 + 16; }

// A dense block of the smoother or of the coarse solve: the velocity slots form
// an nvg x nvg grid of global velocity nodes from (vx0, vy0), the pressure
// slots an npg x npg grid from (px0, py0); pin marks the pressure node (0, 0)
// as pinned (coarse solve).  Slots outside the domain or on the Dirichlet
// boundary are padding (identity rows, zero data).
struct BlockSet {
  int kind;  // 0: one Vanka+star patch per vertex; 1: the single coarse block
  int nvg, npg, ms;  // ms = padded slot count per temporal DoF (leading dimension)
  int local = 0;     // kind 0: 1 = patch system assembled over the patch's own cells
  int weighted = 0;  // kind 0: 1 = scatter weight 1 / (number of patches holding the DoF)
};

FeTables build_tables(int k, int q);
// Largest real part of the eigenvalues of the leading mm x mm block of an upper
// Hessenberg matrix stored row-major with row stride ld (shifted complex QR).
double hessenberg_max_real_eig(const std::vector<double>& H, int mm, int ld);

// ---------------------------------------------------------------- batched launches
// One member of a batched launch at one level depth (0 = every member's finest
// level).  Vectors of all members at a depth live in one arena per role; a
// member's vectors start at `off` (and at `offc` in the next-coarser depth's
// arenas).  The u_* fields are exclusive prefix sums of the work units of the
// members before this one, for each kind of batched kernel; kernels find their
// member by binary search on the prefix that matches their unit.
struct BatchSeg {
  LevelGeom g;           // geometry at this depth
  LevelGeom gc;          // geometry one level coarser (transfers); unused at the coarsest level
  BlockSet bs;           // the patch set (kind 0) or the coarse block (kind 1)
  PhysParams ph;
  int member;
  int64_t off, offc;     // vector offsets at this depth / the next coarser depth
  int64_t off_ye, off_yp;// offsets in the element-contribution and patch-output scratch arenas
  const double* W;       // linearisation point of this level
  const void* factors;   // stored factors of this level (coarse factors for kind 1)
  double* xa;            // absolute right-hand side pointer (coarse-solve tables)
  double* ya;            // absolute output pointer (coarse-solve tables)
  int64_t u_elem, u_dof, u_dofc, u_patch, u_tblk;  // prefixes: element units, DoFs, coarse DoFs, patches, temporal blocks
};

enum BatchUnit { BU_ELEM = 0, BU_DOF = 1, BU_DOFC = 2, BU_PATCH = 3, BU_TBLK = 4 };

// last member whose prefix of `kind` is <= u (members with no units are skipped by construction)
#ifdef __CUDACC__
template <int KIND>
__device__ __forceinline__ int batch_find(const BatchSeg* __restrict__ segs, int nseg, int64_t u) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t b = KIND == BU_ELEM ? segs[mid].u_elem : KIND == BU_DOF ? segs[mid].u_dof
                    : KIND == BU_DOFC ? segs[mid].u_dofc : KIND == BU_PATCH ? segs[mid].u_patch : segs[mid].u_tblk;
    if (b <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}
#endif

// element units of a member level: ceil(cells / 4) x slabs (4 = elements per element-kernel CTA)
inline int64_t elem_units(const LevelGeom& g) { return (int64_t)((g.ncells() + 3) / 4) * g.N; }

// ---------------------------------------------------------------- kernels
void launch_residual(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* U,
                     double* F, double* ye, cudaStream_t s);
void launch_jacobian(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W,
                     const double* x, double* y, double* ye, cudaStream_t s);
// J(W) x with single-precision element arithmetic (FP64 vectors and assembly): the
// smoother's residuals inside the V-cycle of the reduced-precision forms
// W and its reference-cell gradient at the Gauss points of every (cell, slab), the
// input of launch_jacobian_wq (wq_doubles(g) doubles; recomputed at every linearisation)
int64_t wq_doubles(const LevelGeom& g);
void launch_wq(const LevelGeom& g, const FeTables& T, const double* W, double* Wq, cudaStream_t s);
// y = J(W) x from the tabulated W (the solver's form of launch_jacobian)
// (events, if given, are recorded on s around the element kernel alone)
void launch_jacobian_wq(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* Wq,
                        const double* x, double* y, double* ye, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                        cudaEvent_t ev1 = nullptr);
double jac_flops_per_cell_slab(int k, int q);
void launch_jacobian_f32(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W,
                         const double* x, double* y, double* ye, cudaStream_t s);
void launch_boundary_values(const LevelGeom& g, const FeTables& T, const PhysParams& ph, double* U,
                            cudaStream_t s);
// Element convection matrices about W, in FP64 (precision WR_FP64) or FP32 (the
// reduced-precision factorisations, which assemble their blocks in FP32).
void launch_conv_elements(const LevelGeom& g, const FeTables& T, const double* W, void* Ce, int precision,
                          cudaStream_t s);
void launch_inject(const LevelGeom& gf, const LevelGeom& gc, const double* Wf, double* Wc,
                   cudaStream_t s);
// st: a device int of the caller's (zero-pivot flag); with check it is cleared
// before and read back after the launch (a host synchronisation), else left as is.
// Ce: the element convection matrices of launch_conv_elements in the same precision.
void launch_block_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                         const BlockSet& bs, const void* Ce, void* factors, int precision, int* st,
                         cudaStream_t s, bool check = true);
// Patch blocks (kind 0) write [slab][patch][a][slot] outputs to out; the coarse
// block (kind 1) writes the solution.  A window of slabs is g with N = window
// length, r and out offset to the window's first slab, factors of the window,
// and prev = the patch outputs of the slab before it (null: zero jump state).
// Time-parallel split of a patch-block apply (patch blocks only): the items are the
// chunks c_first .. nchunk - 1 of Lc slabs of every block; prev_mode 0: zero jump
// state, 1: chunk c starts from prev + (c - 1) * (one slab of patch outputs), 2: every
// chunk starts from the state prev.
struct ChunkPlan {
  int nchunk = 1, Lc = 0, c_first = 0, prev_mode = 0;
  const double* prev = nullptr;
};
// variant: the apply tile (0 .. 3, -1 = the default of k; patch blocks only), chosen
// per level by the autotuner
void launch_block_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs,
                        const void* factors, int precision, const double* r, double* out,
                        int* err, cudaStream_t s, const double* prev = nullptr, int variant = -1,
                        const ChunkPlan* cp = nullptr);
// Time-parallel patch solve helpers (patch_kernels.cu); mv = 2 nvg^2 velocity slots.
// buf = the state with 1 at velocity slot j of the last temporal DoF of every patch
void cr_unit_state(const LevelGeom& g, const BlockSet& bs, int j, double* buf, cudaStream_t s);
// Tm[(blk, c)][:, j] = the chunk-end velocity state of every chunk in the patch outputs Yp
void cr_gather_column(const LevelGeom& g, const BlockSet& bs, int nchunk, int Lc, int j, const double* Yp,
                      double* Tm, cudaStream_t s);
// carry[c] = e_c + T_c carry[c - 1] for c = 0 .. nchunk - 2 (e_c: chunk-end states in Yp)
void cr_carry(const LevelGeom& g, const BlockSet& bs, int nchunk, int Lc, const double* Tm, const double* Yp,
              double* carry, cudaStream_t s);
constexpr int kApplyTileVariants = 5;
void launch_scatter(const LevelGeom& g, const BlockSet& bs, const double* Yp, double* y,
                    cudaStream_t s);
void launch_restrict(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T,
                     const double* xf, double* xc, cudaStream_t s);
void launch_prolong_add(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T,
                        const double* xc, double* xf, cudaStream_t s);
void launch_project_pressure(const LevelGeom& g, const FeTables& T, double* x, cudaStream_t s);
void launch_zero_dirichlet(const LevelGeom& g, double* x, cudaStream_t s);
void launch_splitmix_free(const LevelGeom& g, uint64_t seed, double* x, cudaStream_t s);

// FP64 vector kernels (deterministic reductions)
void vec_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s);  // y = a x + b y
void vec_axpbypz(int64_t n, double a, const double* x, double b, const double* y, double c, double* z,
                 cudaStream_t s);  // z = a x + b y + c z
void vec_copy(int64_t n, const double* x, double* y, cudaStream_t s);
void vec_scale(int64_t n, double a, double* x, cudaStream_t s);
void vec_zero(int64_t n, double* x, cudaStream_t s);
// dot products into a device scalar; partials must hold dot_partials_size() doubles
int dot_partials_size();
void vec_dot_dev(int64_t n, const double* x, const double* y, double* partials, double* out,
                 cudaStream_t s);
double measure_fp64_tflops(cudaStream_t s);

// Device-resident Krylov scalars (FGMRES and the Arnoldi eigen-estimate).
constexpr int kMaxKrylovBasis = 200;  // largest FGMRES restart length (wr_create refuses more)
struct KrylovBasis {
  const double* p[kMaxKrylovBasis];
};
// w -= (*h) x (skipped if x is null), then *out = <w, y> (deterministic order; one
// launch; partials holds dot_partials_size() doubles, *count is a zeroed counter that
// the launch leaves zeroed)
void krylov_axpy_dot(int64_t n, const double* h, const double* x, double* w, const double* y, double* partials,
                     unsigned* count, double* out, cudaStream_t s);
// w -= (*h) x (skipped if x is null), then *out = ||w|| and *inv = 1 / ||w|| (1 if 0);
// with diag: *inv = 0 where ||w|| <= rel |*diag| + abs (Arnoldi breakdown)
void krylov_axpy_norm(int64_t n, const double* h, const double* x, double* w, double* partials, unsigned* count,
                      double* out, double* inv, const double* diag, double rel, double abs_, cudaStream_t s);
void vec_scale_dev(int64_t n, const double* a, const double* x, double* y, cudaStream_t s);  // y = (*a) x
// the whole MGS column j (w against V.p[0..j], H column col, row stride m, then the
// normalisation; breakdown as in krylov_axpy_norm) in one single-CTA launch, for
// n <= mgs_small_limit()
int64_t mgs_small_limit();
void krylov_mgs_small(int64_t n, const KrylovBasis& V, int j, double* w, double* H, int m, int col, bool breakdown,
                      cudaStream_t s);
// rotations of FGMRES column j (one thread); status[0] = the new residual estimate g[j+1]
void krylov_givens(double* H, double* cs, double* sn, double* g, int j, int m, double* status, cudaStream_t s);
// y = R^{-1} g (leading jend x jend triangle of H), then x += sum_l y_l z_l
void krylov_update(int64_t n, const double* H, const double* g, double* y, int jend, int m, const KrylovBasis& z,
                   double* x, cudaStream_t s);

// batched kernels (one launch for every member in `segs`; base pointers are arenas)
void bt_jacobian(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                 const double* x, double* y, double* ye, cudaStream_t s);
void bt_jacobian_f32(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                     const double* x, double* y, double* ye, cudaStream_t s);
void bt_residual(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                 const double* U, double* F, double* ye, cudaStream_t s);
// coarse_n = 0: patch smoother (scatter into `out`); 2 or 3: coarse block solves of that coarse mesh
void bt_block_apply(int k, int q, int precision, const BatchSeg* segs, int nseg, int64_t items, int64_t dofs,
                    const FeTables& T, const double* r, double* out, double* yp, int* err, int coarse_n,
                    cudaStream_t s, int variant = -1);
void bt_restrict(const BatchSeg* segs, int nseg, int64_t dofsc, const FeTables& T, const double* xf, double* xc,
                 cudaStream_t s);
void bt_prolong_add(const BatchSeg* segs, int nseg, int64_t dofs, const FeTables& T, const double* xc, double* xf,
                    cudaStream_t s);
void bt_project_pressure(const BatchSeg* segs, int nseg, int64_t tblks, const FeTables& T, double* x, bool absolute,
                         cudaStream_t s);
void bt_splitmix(const BatchSeg* segs, int nseg, int64_t dofs, const int64_t* seeds, double* x, cudaStream_t s);
void bt_boundary(const BatchSeg* segs, int nseg, int64_t dofs, const FeTables& T, double* U, cudaStream_t s);
// y = a_m x + b_m y per member (a_m, b_m device arrays indexed by segment, or scalars if null)
void bt_axpby(const BatchSeg* segs, int nseg, int64_t dofs, const double* a, double as, const double* x,
              const double* b, double bs_, double* y, cudaStream_t s);
void bt_copy(const BatchSeg* segs, int nseg, int64_t dofs, const double* x, double* y, cudaStream_t s);
// per-member dot products into out[nseg]; partials holds nseg * bt_dot_blocks() doubles
// segs[m].ya[i] = v for i < segs[m].g.ndofs (absolute pointers; BU_DOF prefix)
void bt_fill_abs(const BatchSeg* segs, int nseg, int64_t dofs, double v, cudaStream_t s);
int bt_dot_blocks();
void bt_dot(const BatchSeg* segs, int nseg, const double* x, const double* y, double* partials, double* out,
            cudaStream_t s);

// Batched Krylov scalars, member-indexed (array of member b at base + b * stride):
// w -= h_b x (if hoff >= 0, h_b = hbase[b * hstride + hoff]) and out[b * ostride + ooff] = <w, y>
void bt_axpy_dot(const BatchSeg* segs, int nseg, const double* hbase, int64_t hstride, int hoff, const double* x,
                 double* w, const double* y, double* partials, double* out, int64_t ostride, int ooff,
                 cudaStream_t s);
// the same update, then out[...] = ||w||, inv[b] = 1 / ||w|| (1 if 0; with doff >= 0, 0
// where ||w|| <= 1e-14 |out[b * ostride + doff]| + 1e-300), g[b * gstride] = ||w|| if g
void bt_axpy_norm(const BatchSeg* segs, int nseg, const double* hbase, int64_t hstride, int hoff, const double* x,
                  double* w, double* partials, double* out, int64_t ostride, int ooff, double* inv, int doff,
                  double* g, int64_t gstride, cudaStream_t s);
void bt_scale_dev(const BatchSeg* segs, int nseg, int64_t dofs, const double* a, const double* x, double* y,
                  cudaStream_t s);  // y = a_b x
// FGMRES column j of every member (H: (R+1) x R, cs, sn: R, g: R+1 per member); status[seg]
void bt_givens(const BatchSeg* segs, int nseg, double* H, double* cs, double* sn, double* g, int R, int j,
               double* status, cudaStream_t s);
void bt_krylov_update(const BatchSeg* segs, int nseg, int64_t dofs, const double* H, const double* g, double* y, int R,
                      int jend, const KrylovBasis& z, double* x, cudaStream_t s);

// wr_create with the option of allocating the context's device memory from the
// stream-ordered pool on `stream` (cudaMallocAsync / cudaFreeAsync), so that
// creating and destroying a context never synchronises the whole device while
// other streams run.
int create_context(wr_ctx** out, const wr_problem* p, const wr_options* o, void* stream, bool stream_ordered);

// wr_batch_solve with per-member completion: as soon as member m leaves the lock-step
// set (converged, gave up, failed, or cancelled through cancel[m]) its iterate is
// copied to U[m], st[m] is final and on_done(m, status) runs on the calling thread.
int batch_solve_hooked(wr_batch* b, double* const* U, wr_stats* st, const std::atomic<int>* const* cancel,
                       const std::function<void(int, int)>& on_done);

// The apply kernels' bounded wait on an mbarrier that never completes: *timed_out = 1
// and *ns = the time waited (device pointers).
void launch_bounded_wait_selftest(int* timed_out, unsigned long long* ns, cudaStream_t s);

// The server's per-request cancel flag: the context's solve stops with
// WR_ERR_CANCELLED at its next Newton step or FGMRES iteration once it is set.
void set_cancel_flag(wr_ctx* c, const std::atomic<int>* flag);
// Host-side fault injection counter (wr_inject_alloc_failure).
extern std::atomic<int64_t> g_fail_alloc;

// Key of a tuned smoother-apply tile: kind (0 context level, 1 batch depth), k, q,
// precision, blocks per launch, slabs.
struct TuneKey {
  int kind, k, q, precision;
  int64_t blocks;
  int slabs;
  bool operator<(const TuneKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (k != o.k) return k < o.k;
    if (q != o.q) return q < o.q;
    if (precision != o.precision) return precision < o.precision;
    if (blocks != o.blocks) return blocks < o.blocks;
    return slabs < o.slabs;
  }
};
int tune_apply_variant(const TuneKey& key, cudaStream_t s, const std::function<void(int)>& launch);

// ---------------------------------------------------------------- heat equation (heat.cu)
LevelGeom make_heat_geom(int n, int k, int q, int N, double T);
int heat_block_size(int k, int q, int n_whole);  // slots per (block, slab): (q+1) PX^2; n_whole = 0: a patch
bool heat_block_fits(int k, int q, int n_whole);  // the block's FP64 inversion fits in shared memory
// y = J x and F(x) by tensor-product passes; tmp: heat_op_scratch(g) doubles of device scratch
size_t heat_op_scratch(const LevelGeom& g);
void heat_jacobian(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* x, double* y,
                   double* tmp, cudaStream_t s);
void heat_residual(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* x, double* y,
                   double* tmp, cudaStream_t s);
// inverts every (patch, slab) block (coarse: the single whole-mesh block); st as in launch_block_factor
void heat_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph, bool coarse, double* f, int* st,
                 cudaStream_t s);
void heat_patch_apply(const LevelGeom& g, const FeTables& T, const double* f, const double* r, double* Yp, double* y,
                      cudaStream_t s);
void heat_coarse_apply(const LevelGeom& g, const FeTables& T, const double* f, const double* b, double* x,
                       cudaStream_t s);
void heat_restrict(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xf, double* xc,
                   cudaStream_t s);
void heat_prolong_add(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xc, double* xf,
                      cudaStream_t s);
void heat_splitmix(int64_t n, uint64_t seed, double* x, cudaStream_t s);
// slot -> node index (-1 outside the domain) of heat patch blk into d_out; returns the slot count
int heat_patch_slots(const LevelGeom& g, int blk, int* d_out, cudaStream_t s);
