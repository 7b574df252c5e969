// Internal declarations shared by the translation units of libwrmg.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "wrmg.h"

#ifdef __CUDACC__
#define WR_HD __host__ __device__
#else
#define WR_HD
#endif

// Compile-time bounds: k <= 2 (Q3/Q2), q <= 1 (DG(1)).
#define WR_MAX_NQ 5   // Gauss points per direction, k + 3
#define WR_MAX_NVL 4  // velocity nodes per cell and direction, k + 2
#define WR_MAX_NPL 3  // pressure nodes per cell and direction, k + 1
#define WR_MAX_NT 2   // temporal DoFs per slab, q + 1
#define WR_MAX_NTQ 3  // Gauss points in time for the forcing, q + 2

struct WrError : std::runtime_error {
  int code;
  WrError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define WR_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw WrError(e_ == cudaErrorMemoryAllocation ? WR_ERR_NOMEM : WR_ERR_CUDA,       \
                    std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)
// Every kernel launch of the library is followed by WR_LAUNCH_CHECK, which also counts it.
void wr_count_launch();
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
inline int64_t factor_block_elems(int k, int precision) {
  const int64_t e = (int64_t)patch_ms(k) * patch_ms(k);
  const int64_t g = precision == WR_FP32 ? 4 : 2;
  return (e + g - 1) / g * g;
}

// A dense block of the smoother or of the coarse solve: the velocity slots form
// an nvg x nvg grid of global velocity nodes from (vx0, vy0), the pressure
// slots an npg x npg grid from (px0, py0); pin marks the pressure node (0, 0)
// as pinned (coarse solve).  Slots outside the domain or on the Dirichlet
// boundary are padding (identity rows, zero data).
struct BlockSet {
  int kind;  // 0: one Vanka+star patch per vertex; 1: the single coarse block
  int nvg, npg, ms;  // ms = padded slot count per temporal DoF (leading dimension)
};

FeTables build_tables(int k, int q);

// ---------------------------------------------------------------- kernels
void launch_residual(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* U,
                     double* F, double* ye, cudaStream_t s);
void launch_jacobian(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W,
                     const double* x, double* y, double* ye, cudaStream_t s);
void launch_boundary_values(const LevelGeom& g, const FeTables& T, const PhysParams& ph, double* U,
                            cudaStream_t s);
void launch_conv_elements(const LevelGeom& g, const FeTables& T, const double* W, double* Ce,
                          cudaStream_t s);
void launch_inject(const LevelGeom& gf, const LevelGeom& gc, const double* Wf, double* Wc,
                   cudaStream_t s);
void launch_block_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                         const BlockSet& bs, const double* Ce, void* factors, int precision,
                         cudaStream_t s);
void launch_block_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs,
                        const void* factors, int precision, const double* r, double* out,
                        int* err, cudaStream_t s);
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
