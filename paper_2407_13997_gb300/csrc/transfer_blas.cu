// Grid transfers (hot-path step (f)), pressure-mean projection, FP64 vector
// kernels with deterministic reductions, and the FP64 throughput probe.
//
// Transfers (Sec. 3): P = I_t (x) blockdiag(P_u, P_phi), R = P^T, with
// P_u = P1_v (x) P1_v per velocity component and P_phi = P1_p (x) P1_p, where
// P1[f, c] is the coarse 1D Lagrange basis function c at fine node f.  Fine node
// f lies in coarse cell min(f / 2p, nc - 1) at offset r = f - 2p cell, and its
// weights on the coarse cell's p+1 nodes are the tabulated phi_l(r / 2p).
// Dirichlet velocity rows and columns are zero (corrections vanish there).
#include <cmath>

#include "wrmg_internal.h"

namespace {

// weight of coarse node ic at fine node f (1D, degree p, nc coarse cells)
__device__ __forceinline__ double w1d(const double* tab, int ld, int p, int nc, int f, int ic) {
  const int c = min(f / (2 * p), nc - 1);
  const int l = ic - p * c;
  if (l < 0 || l > p) return 0.0;
  return tab[(f - 2 * p * c) * ld + l];
}

__device__ __forceinline__ void prolong_body(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T,
                                             const double* __restrict__ xc, double* __restrict__ xf, int64_t idx) {
  const int64_t blk = idx / gf.S;
  const int sp = int(idx % gf.S);
  const int nvf2 = gf.nv * gf.nv, nvc2 = gc.nv * gc.nv;
  const double* xcb = xc + blk * gc.S;
  double acc = 0.0;
  if (sp < 2 * nvf2) {
    const int c = sp / nvf2, t = sp % nvf2, fx = t % gf.nv, fy = t / gf.nv;
    if (fx == 0 || fy == 0 || fx == gf.nv - 1 || fy == gf.nv - 1) return;  // Dirichlet: P row is zero
    const int p = gf.k + 1, nc = gc.n;
    const int cx = min(fx / (2 * p), nc - 1), cy = min(fy / (2 * p), nc - 1);
    const double* tx = T.pv[fx - 2 * p * cx];
    const double* ty = T.pv[fy - 2 * p * cy];
    for (int ly = 0; ly <= p; ++ly) {
      const int Y = p * cy + ly;
      if (ty[ly] == 0.0 || Y == 0 || Y == gc.nv - 1) continue;
      for (int lx = 0; lx <= p; ++lx) {
        const int X = p * cx + lx;
        if (tx[lx] == 0.0 || X == 0 || X == gc.nv - 1) continue;
        acc = fma(ty[ly] * tx[lx], xcb[c * nvc2 + Y * gc.nv + X], acc);
      }
    }
  } else {
    const int t = sp - 2 * nvf2, fx = t % gf.np, fy = t / gf.np;
    const int p = gf.k, nc = gc.n;
    const int cx = min(fx / (2 * p), nc - 1), cy = min(fy / (2 * p), nc - 1);
    const double* tx = T.pp[fx - 2 * p * cx];
    const double* ty = T.pp[fy - 2 * p * cy];
    for (int ly = 0; ly <= p; ++ly) {
      if (ty[ly] == 0.0) continue;
      for (int lx = 0; lx <= p; ++lx) {
        if (tx[lx] == 0.0) continue;
        acc = fma(ty[ly] * tx[lx], xcb[2 * nvc2 + (p * cy + ly) * gc.np + p * cx + lx], acc);
      }
    }
  }
  xf[idx] += acc;
}

__global__ void prolong_add_kernel(LevelGeom gf, LevelGeom gc, FeTables T, const double* __restrict__ xc,
                                   double* __restrict__ xf) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= gf.ndofs) return;
  prolong_body(gf, gc, T, xc, xf, idx);
}

__device__ __forceinline__ void restrict_body(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T,
                                              const double* __restrict__ xf, double* __restrict__ xc, int64_t idx) {
  const int64_t blk = idx / gc.S;
  const int sp = int(idx % gc.S);
  const int nvf2 = gf.nv * gf.nv, nvc2 = gc.nv * gc.nv;
  const double* xfb = xf + blk * gf.S;
  double acc = 0.0;
  if (sp < 2 * nvc2) {
    const int c = sp / nvc2, t = sp % nvc2, X = t % gc.nv, Y = t / gc.nv;
    if (X == 0 || Y == 0 || X == gc.nv - 1 || Y == gc.nv - 1) { xc[idx] = 0.0; return; }
    const int p = gf.k + 1, nc = gc.n;
    // fine nodes in the coarse cells around X (support of the coarse basis function)
    const int fx0 = 2 * p * max(0, (X - 1) / p), fx1 = min(2 * p * (min(X / p, nc - 1) + 1), gf.nv - 1);
    const int fy0 = 2 * p * max(0, (Y - 1) / p), fy1 = min(2 * p * (min(Y / p, nc - 1) + 1), gf.nv - 1);
    for (int fy = max(fy0, 1); fy <= min(fy1, gf.nv - 2); ++fy) {
      const double wy = w1d(&T.pv[0][0], WR_MAX_NVL, p, nc, fy, Y);
      if (wy == 0.0) continue;
      for (int fx = max(fx0, 1); fx <= min(fx1, gf.nv - 2); ++fx) {
        const double wx = w1d(&T.pv[0][0], WR_MAX_NVL, p, nc, fx, X);
        if (wx == 0.0) continue;
        acc = fma(wy * wx, xfb[c * nvf2 + fy * gf.nv + fx], acc);
      }
    }
  } else {
    const int t = sp - 2 * nvc2, X = t % gc.np, Y = t / gc.np;
    const int p = gf.k, nc = gc.n;
    const int fx0 = 2 * p * max(0, (X - 1) / p), fx1 = min(2 * p * (min(X / p, nc - 1) + 1), gf.np - 1);
    const int fy0 = 2 * p * max(0, (Y - 1) / p), fy1 = min(2 * p * (min(Y / p, nc - 1) + 1), gf.np - 1);
    for (int fy = fy0; fy <= fy1; ++fy) {
      const double wy = w1d(&T.pp[0][0], WR_MAX_NPL, p, nc, fy, Y);
      if (wy == 0.0) continue;
      for (int fx = fx0; fx <= fx1; ++fx) {
        const double wx = w1d(&T.pp[0][0], WR_MAX_NPL, p, nc, fx, X);
        if (wx == 0.0) continue;
        acc = fma(wy * wx, xfb[2 * nvf2 + fy * gf.np + fx], acc);
      }
    }
  }
  xc[idx] = acc;
}

__global__ void restrict_kernel(LevelGeom gf, LevelGeom gc, FeTables T, const double* __restrict__ xf,
                                double* __restrict__ xc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= gc.ndofs) return;
  restrict_body(gf, gc, T, xf, xc, idx);
}

// ---------------------------------------------------------------- tiled tensor-product transfers
// R = P^T and P applied per field as two 1D passes (x, then y) over a tile held in
// shared memory.  The equispaced nodes are nested: fine node 2C is coarse node C, and
// the fine nodes strictly inside a coarse cell (odd local index r) carry the degree-p
// Lagrange weights pv[r][l] of the cell's p+1 coarse nodes.  So coarse node C takes
// fine node 2C with weight 1 plus the 2p odd nodes of its (at most two) cells, and a
// fine node takes either one coarse value (even r) or p+1 weighted ones (odd r).
// Velocity Dirichlet nodes are zero on both sides, as in the oracle's P.
constexpr int kTrBX = 32, kTrBY = 16;  // restriction: coarse nodes per tile (x, y)
constexpr int kTpBX = 64, kTpBY = 32;  // prolongation: fine nodes per tile (x, y)

template <int P>
__device__ __forceinline__ int tr_cell_lo(int C) { return C == 0 ? 0 : (C - 1) / P; }

// sum over the 1D support of coarse node C of wts(f, C) v(f), f fine (coincident + odd)
template <int P, int LD, class V>
__device__ __forceinline__ double tr_restrict_1d(const double (*pv)[LD], int nc, int C, V v) {
  double acc = v(2 * C);
  const int c0 = tr_cell_lo<P>(C), c1 = min(C / P, nc - 1);
  for (int cc = c0; cc <= c1; ++cc) {
    const int l = C - P * cc;
#pragma unroll
    for (int r = 1; r < 2 * P; r += 2) acc = fma(pv[r][l], v(2 * P * cc + r), acc);
  }
  return acc;
}

// value at fine node f of the coarse interpolant of u
template <int P, int LD, class U>
__device__ __forceinline__ double tr_prolong_1d(const double (*pv)[LD], int nc, int f, U u) {
  const int cc = min(f / (2 * P), nc - 1), r = f - 2 * P * cc;
  if ((r & 1) == 0) return u(P * cc + r / 2);
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l <= P; ++l) acc = fma(pv[r][l], u(P * cc + l), acc);
  return acc;
}

template <int P, bool VEL, int LD>
__device__ void restrict_tile(const double (*pv)[LD], int ncf, const double* __restrict__ xf,
                              double* __restrict__ xc, double* smem) {
  const int nc = ncf / 2, nvf = ncf * P + 1, nvc = nc * P + 1;
  const int X0 = blockIdx.x * kTrBX, Y0 = blockIdx.y * kTrBY;
  if (X0 >= nvc || Y0 >= nvc) return;
  const int X1 = min(X0 + kTrBX, nvc), Y1 = min(Y0 + kTrBY, nvc);
  const int fx0 = 2 * P * tr_cell_lo<P>(X0), fx1 = min(2 * P * (min((X1 - 1) / P, nc - 1) + 1), nvf - 1);
  const int fy0 = 2 * P * tr_cell_lo<P>(Y0), fy1 = min(2 * P * (min((Y1 - 1) / P, nc - 1) + 1), nvf - 1);
  const int W = fx1 - fx0 + 1, H = fy1 - fy0 + 1, BW = X1 - X0;
  double* tf = smem;        // fine tile, H x W
  double* tt = smem + H * W;  // after the x pass, H x BW
  for (int e = threadIdx.x; e < H * W; e += blockDim.x) {
    const int fy = fy0 + e / W, fx = fx0 + e % W;
    const bool dir = VEL && (fx == 0 || fy == 0 || fx == nvf - 1 || fy == nvf - 1);
    tf[e] = dir ? 0.0 : xf[(int64_t)fy * nvf + fx];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < H * BW; e += blockDim.x) {
    const int row = e / BW, X = X0 + e % BW;
    const double* rowp = tf + row * W - fx0;
    tt[e] = tr_restrict_1d<P, LD>(pv, nc, X, [&](int f) { return rowp[f]; });
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (Y1 - Y0) * BW; e += blockDim.x) {
    const int Y = Y0 + e / BW, xi = e % BW, X = X0 + xi;
    double v = tr_restrict_1d<P, LD>(pv, nc, Y, [&](int f) { return tt[(f - fy0) * BW + xi]; });
    if (VEL && (X == 0 || Y == 0 || X == nvc - 1 || Y == nvc - 1)) v = 0.0;
    xc[(int64_t)Y * nvc + X] = v;
  }
}

template <int P, bool VEL, int LD>
__device__ void prolong_tile(const double (*pv)[LD], int ncf, const double* __restrict__ xc,
                             double* __restrict__ xf, double* smem) {
  const int nc = ncf / 2, nvf = ncf * P + 1, nvc = nc * P + 1;
  const int F0x = blockIdx.x * kTpBX, F0y = blockIdx.y * kTpBY;
  if (F0x >= nvf || F0y >= nvf) return;
  const int F1x = min(F0x + kTpBX, nvf), F1y = min(F0y + kTpBY, nvf);
  const int cx0 = P * min(F0x / (2 * P), nc - 1), cx1 = P * min((F1x - 1) / (2 * P), nc - 1) + P;
  const int cy0 = P * min(F0y / (2 * P), nc - 1), cy1 = P * min((F1y - 1) / (2 * P), nc - 1) + P;
  const int W = cx1 - cx0 + 1, H = cy1 - cy0 + 1, FW = F1x - F0x;
  double* tc = smem;          // coarse tile, H x W
  double* tt = smem + H * W;  // after the x pass, H x FW
  for (int e = threadIdx.x; e < H * W; e += blockDim.x) {
    const int Y = cy0 + e / W, X = cx0 + e % W;
    const bool dir = VEL && (X == 0 || Y == 0 || X == nvc - 1 || Y == nvc - 1);
    tc[e] = dir ? 0.0 : xc[(int64_t)Y * nvc + X];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < H * FW; e += blockDim.x) {
    const int row = e / FW, fx = F0x + e % FW;
    const double* rowp = tc + row * W - cx0;
    tt[e] = tr_prolong_1d<P, LD>(pv, nc, fx, [&](int C) { return rowp[C]; });
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (F1y - F0y) * FW; e += blockDim.x) {
    const int fy = F0y + e / FW, xi = e % FW, fx = F0x + xi;
    if (VEL && (fx == 0 || fy == 0 || fx == nvf - 1 || fy == nvf - 1)) continue;  // P row is zero
    xf[(int64_t)fy * nvf + fx] += tr_prolong_1d<P, LD>(pv, nc, fy, [&](int C) { return tt[(C - cy0) * FW + xi]; });
  }
}

// grid: (x tiles, y tiles, temporal blocks x 3 fields); the fields u_x, u_y (degree
// k+1, Dirichlet) and the pressure (degree k) of one temporal block
template <int K>
__global__ void __launch_bounds__(256) restrict_tiled_kernel(LevelGeom gf, LevelGeom gc,
                                                             const __grid_constant__ FeTables T,
                                                             const double* __restrict__ xf,
                                                             double* __restrict__ xc) {
  extern __shared__ double trs[];
  const int64_t blk = blockIdx.z / 3;
  const int field = blockIdx.z % 3;
  const int64_t nvf2 = (int64_t)gf.nv * gf.nv, nvc2 = (int64_t)gc.nv * gc.nv;
  const double* src = xf + blk * gf.S;
  double* dst = xc + blk * gc.S;
  if (field < 2) restrict_tile<K + 1, true>(T.pv, gf.n, src + field * nvf2, dst + field * nvc2, trs);
  else restrict_tile<K, false>(T.pp, gf.n, src + 2 * nvf2, dst + 2 * nvc2, trs);
}

template <int K>
__global__ void __launch_bounds__(256) prolong_tiled_kernel(LevelGeom gf, LevelGeom gc,
                                                            const __grid_constant__ FeTables T,
                                                            const double* __restrict__ xc,
                                                            double* __restrict__ xf) {
  extern __shared__ double trs[];
  const int64_t blk = blockIdx.z / 3;
  const int field = blockIdx.z % 3;
  const int64_t nvf2 = (int64_t)gf.nv * gf.nv, nvc2 = (int64_t)gc.nv * gc.nv;
  const double* src = xc + blk * gc.S;
  double* dst = xf + blk * gf.S;
  if (field < 2) prolong_tile<K + 1, true>(T.pv, gf.n, src + field * nvc2, dst + field * nvf2, trs);
  else prolong_tile<K, false>(T.pp, gf.n, src + 2 * nvc2, dst + 2 * nvf2, trs);
}

// Pressure weight int chi_j of node g in 1D: h sum over cells containing g of mp1.
__device__ __forceinline__ double pw1(const FeTables& T, int k, int n, double h, int g) {
  const int lo = g == 0 ? 0 : (g - 1) / k, hi = min(g / k, n - 1);
  double v = 0.0;
  for (int c = lo; c <= hi; ++c) v += T.mp1[g - k * c];
  return h * v;
}

// One CTA per temporal block: Phi -= (sum_j w_j Phi_j) / (sum_j w_j), fixed-order reduction.
__device__ __forceinline__ void project_body(const LevelGeom& g, const FeTables& T, double* __restrict__ x,
                                             int64_t tblk) {
  __shared__ double sa[256], sb[256];
  double* p = x + tblk * g.S + 2 * g.nv * g.nv;
  const int np2 = g.np * g.np;
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < np2; j += blockDim.x) {
    const double w = pw1(T, g.k, g.n, g.h, j % g.np) * pw1(T, g.k, g.n, g.h, j / g.np);
    a = fma(w, p[j], a);
    b += w;
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  const double mean = sa[0] / sb[0];
  for (int j = threadIdx.x; j < np2; j += blockDim.x) p[j] -= mean;
}

__global__ void project_pressure_kernel(LevelGeom g, FeTables T, double* __restrict__ x) {
  project_body(g, T, x, blockIdx.x);
}

__global__ void zero_dirichlet_kernel(LevelGeom g, double* __restrict__ x) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  const int sp = int(idx % g.S), nv = g.nv, nv2 = nv * nv;
  if (sp < 2 * nv2) {
    const int t = sp % nv2, gx = t % nv, gy = t / nv;
    if (gx == 0 || gy == 0 || gx == nv - 1 || gy == nv - 1) x[idx] = 0.0;
  }
}

// uniform(-1, 1) from splitmix64 (Steele, Lea & Flood 2014), counter-based:
// value i = mix(seed + (i+1) * 0x9E3779B97F4A7C15), top 53 bits; zero on Dirichlet DoFs.
__global__ void splitmix_kernel(LevelGeom g, uint64_t seed, double* __restrict__ x) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  uint64_t z = seed + (uint64_t)(idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  u = 2.0 * u - 1.0;
  const int sp = int(idx % g.S), nv = g.nv, nv2 = nv * nv;
  if (sp < 2 * nv2) {
    const int t = sp % nv2, gx = t % nv, gy = t / nv;
    if (gx == 0 || gy == 0 || gx == nv - 1 || gy == nv - 1) u = 0.0;
  }
  x[idx] = u;
}

__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}
__global__ void axpbypz_kernel(int64_t n, double a, const double* __restrict__ x, double b,
                               const double* __restrict__ y, double c, double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = fma(a, x[i], fma(b, y[i], c * z[i]));
}
__global__ void copy_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}
__global__ void scale_kernel(int64_t n, double a, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

constexpr int kDotBlocks = 1024, kDotThreads = 256;

// Deterministic dot: each block sums a fixed strided set in a fixed tree, then one block sums the partials.
__global__ void dot_stage1(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                           double* __restrict__ partials) {
  __shared__ double s[kDotThreads];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
    a = fma(x[i], y[i], a);
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kDotThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}
__global__ void dot_stage2(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double s[kDotThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) a += partials[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kDotThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ---------------------------------------------------------------- device-resident Krylov scalars
// FGMRES and the Arnoldi eigen-estimate keep every Hessenberg entry, Givens rotation
// and least-squares coefficient in device memory (FP64); the host reads one status
// word per FGMRES iteration.  Modified Gram-Schmidt keeps its order: step i updates
// w -= h_{i-1} v_{i-1} with the coefficient the previous step left on the device and
// forms <w, v_i> in the same pass.  One launch per step: every block writes its partial
// sum (a fixed strided set, a fixed tree), and the last block to finish sums the
// partials in a fixed order, so the result depends on n only, not on block timing.
// The grid is sized from n (at least 4 elements per thread, at most kDotBlocks).
inline int krylov_blocks(int64_t n) {
  const int64_t b = (n + 4 * kDotThreads - 1) / (4 * kDotThreads);
  return (int)(b < 1 ? 1 : b > kDotBlocks ? kDotBlocks : b);
}

// mode 0: *out = <w, y>.  mode 1 (a norm, y = w): *out = ||w|| and *inv = 1 / *out (1 if
// *out is 0).  mode 2 (Arnoldi with a breakdown test): *out = ||w||, *inv = 1 / *out
// unless *out <= rel |*diag| + abs, where it is 0 (the basis ends there; later vectors
// are zero).  *count must be 0 before the launch; the last block resets it.
__global__ void axpy_dot_kernel(int64_t n, const double* __restrict__ h, const double* __restrict__ x, double* w,
                                const double* y, double* __restrict__ partials, unsigned* __restrict__ count,
                                double* __restrict__ out, int mode, double* __restrict__ inv,
                                const double* __restrict__ diag, double rel, double abs_) {
  __shared__ double s[kDotThreads];
  __shared__ bool last;
  const double a = x ? -*h : 0.0;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
    double wi = w[i];
    if (x) {
      wi = fma(a, x[i], wi);
      w[i] = wi;
    }
    acc = fma(wi, y == w ? wi : y[i], acc);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int st = kDotThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s[0];
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double b = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kDotThreads) b += __ldcg(partials + i);
  s[threadIdx.x] = b;
  __syncthreads();
  for (int st = kDotThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *count = 0u;
    if (mode == 0) {
      *out = s[0];
      return;
    }
    const double hn = sqrt(s[0]);
    *out = hn;
    if (mode == 1) *inv = hn != 0.0 ? 1.0 / hn : 1.0;
    else *inv = hn > rel * fabs(*diag) + abs_ ? 1.0 / hn : 0.0;
  }
}

// A whole modified Gram-Schmidt column in one launch, for short vectors (one CTA):
// for i = 0..j in order, H[i m + col] = <w, v_i> and w -= H[i m + col] v_i; then
// H[(j+1) m + col] = ||w|| and w /= ||w|| (mode 1: unless 0; mode 2: w = 0 where
// ||w|| <= rel |H[j m + col]| + abs, the Arnoldi breakdown).  Every thread owns the same
// strided elements in every pass, so w needs no barrier; the sums are fixed trees.
constexpr int kMgsThreads = 256;
// Sum over the CTA in a fixed order: a butterfly in each warp (lane 0's result), then
// one warp over the warps' sums; every thread gets the total.
__device__ __forceinline__ double block_sum_fixed(double a, double* s) {
  constexpr int NW = kMgsThreads / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if (lane == 0) s[wid] = a;
  __syncthreads();
  if (wid == 0) {
    double b = lane < NW ? s[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) b += __shfl_xor_sync(0xffffffffu, b, off);
    if (lane == 0) s[NW] = b;
  }
  __syncthreads();
  return s[NW];
}
__global__ void __launch_bounds__(kMgsThreads)
mgs_small_kernel(int64_t n, KrylovBasis V, int j, double* __restrict__ w, double* __restrict__ H, int m, int col,
                 int mode, double rel, double abs_) {
  __shared__ double s[kMgsThreads / 32 + 1];
  for (int i = 0; i <= j; ++i) {
    const double* __restrict__ v = V.p[i];
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < n; t += kMgsThreads) acc = fma(w[t], v[t], acc);
    const double h = block_sum_fixed(acc, s);
    if (threadIdx.x == 0) H[i * m + col] = h;
    for (int64_t t = threadIdx.x; t < n; t += kMgsThreads) w[t] = fma(-h, v[t], w[t]);
  }
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += kMgsThreads) acc = fma(w[t], w[t], acc);
  const double hn = sqrt(block_sum_fixed(acc, s));
  double inv;
  if (mode == 1) inv = hn != 0.0 ? 1.0 / hn : 1.0;
  else inv = hn > rel * fabs(H[j * m + col]) + abs_ ? 1.0 / hn : 0.0;
  if (threadIdx.x == 0) H[(j + 1) * m + col] = hn;
  for (int64_t t = threadIdx.x; t < n; t += kMgsThreads) w[t] *= inv;
}

// y = a x with the scalar a in device memory (y may be x)
__global__ void scale_dev_kernel(int64_t n, const double* __restrict__ a, const double* x, double* y) {
  const double av = *a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * av;
}

// One FGMRES iteration's least-squares update (one thread): the earlier rotations
// applied to column j of H (row stride m), the new rotation that zeroes H[j+1][j],
// and the rotated right-hand side g; status[0] = g[j+1] (the residual estimate).
__global__ void givens_kernel(double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, int j, int m, double* __restrict__ status) {
  for (int i = 0; i < j; ++i) {
    const double hi = H[i * m + j], hi1 = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * hi + sn[i] * hi1;
    H[(i + 1) * m + j] = -sn[i] * hi + cs[i] * hi1;
  }
  const double a = H[j * m + j], b = H[(j + 1) * m + j];
  const double den = hypot(a, b);
  cs[j] = a / den;
  sn[j] = b / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  status[0] = g[j + 1];
}

// Back substitution R y = g for the leading jend x jend upper triangle of H (one thread).
__global__ void trisolve_kernel(const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y,
                                int jend, int m) {
  for (int i = jend - 1; i >= 0; --i) {
    double acc = g[i];
    for (int l = i + 1; l < jend; ++l) acc -= H[i * m + l] * y[l];
    y[i] = acc / H[i * m + i];
  }
}

// x += sum_l y_l Z_l, the terms added one after another (the order of separate updates)
__global__ void multi_axpy_kernel(int64_t n, const double* __restrict__ y, KrylovBasis z, int cnt,
                                  double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xi = x[i];
    for (int l = 0; l < cnt; ++l) xi = fma(y[l], z.p[l][i], xi);
    x[i] = xi;
  }
}

// 8 independent FMA chains per thread, register only.
__global__ void fp64_probe_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// ---------------------------------------------------------------- batched variants
__global__ void bt_restrict_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofsc, FeTables T,
                                   const double* __restrict__ xf, double* __restrict__ xc) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofsc) return;
  const int m = batch_find<BU_DOFC>(segs, nseg, u);
  const LevelGeom gf = segs[m].g, gc = segs[m].gc;
  restrict_body(gf, gc, T, xf + segs[m].off, xc + segs[m].offc, u - segs[m].u_dofc);
}
__global__ void bt_prolong_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, FeTables T,
                                  const double* __restrict__ xc, double* __restrict__ xf) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const LevelGeom gf = segs[m].g, gc = segs[m].gc;
  prolong_body(gf, gc, T, xc + segs[m].offc, xf + segs[m].off, u - segs[m].u_dof);
}
__global__ void bt_project_kernel(const BatchSeg* __restrict__ segs, int nseg, FeTables T, double* __restrict__ x,
                                  int absolute) {
  const int m = batch_find<BU_TBLK>(segs, nseg, blockIdx.x);
  const LevelGeom g = segs[m].g;
  double* base = absolute ? segs[m].ya : x + segs[m].off;
  project_body(g, T, base, blockIdx.x - segs[m].u_tblk);
}
__global__ void bt_splitmix_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs,
                                   const int64_t* __restrict__ seeds, double* __restrict__ x) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const LevelGeom g = segs[m].g;
  const int64_t idx = u - segs[m].u_dof;
  uint64_t z = (uint64_t)seeds[m] + (uint64_t)(idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double v = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  const int sp = int(idx % g.S), nv = g.nv, nv2 = nv * nv;
  if (sp < 2 * nv2) {
    const int t = sp % nv2, gx = t % nv, gy = t / nv;
    if (gx == 0 || gy == 0 || gx == nv - 1 || gy == nv - 1) v = 0.0;
  }
  x[segs[m].off + idx] = v;
}
__global__ void bt_axpby_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, const double* __restrict__ a,
                                double as, const double* __restrict__ x, const double* __restrict__ b, double bs_,
                                double* __restrict__ y) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const int64_t i = segs[m].off + (u - segs[m].u_dof);
  const double am = a ? a[m] : as, bm = b ? b[m] : bs_;
  y[i] = fma(am, x[i], bm * y[i]);
}
__global__ void bt_copy_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, const double* __restrict__ x,
                               double* __restrict__ y) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const int64_t i = segs[m].off + (u - segs[m].u_dof);
  y[i] = x[i];
}
__global__ void bt_fill_abs_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, double v) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  segs[m].ya[u - segs[m].u_dof] = v;
}
constexpr int kBtDotBlocks = 64;
// grid (kBtDotBlocks, nseg): fixed strided partial sums per member, then a fixed tree
__global__ void bt_dot_stage1(const BatchSeg* __restrict__ segs, const double* __restrict__ x,
                              const double* __restrict__ y, double* __restrict__ partials) {
  __shared__ double sbuf[256];
  const int m = blockIdx.y;
  const int64_t n = segs[m].g.ndofs, off = segs[m].off;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kBtDotBlocks * 256)
    acc = fma(x[off + i], y[off + i], acc);
  sbuf[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sbuf[threadIdx.x] += sbuf[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[m * kBtDotBlocks + blockIdx.x] = sbuf[0];
}
__global__ void bt_dot_stage2(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sbuf[64];
  const int m = blockIdx.x;
  sbuf[threadIdx.x] = partials[m * kBtDotBlocks + threadIdx.x];
  __syncthreads();
  for (int st = 32; st > 0; st >>= 1) {
    if (threadIdx.x < st) sbuf[threadIdx.x] += sbuf[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[m] = sbuf[0];
}

// ---- batched Krylov scalars on the device, member-indexed (member = segs[seg].member):
// the FGMRES/Arnoldi arrays of member b start at base + b * stride.
// MGS step of every member: w -= h_b x (if hoff >= 0, h_b = hbase[b * hstride + hoff]),
// then the partial sums of <w, y> in bt_dot_stage1's pattern and order.
__global__ void bt_axpy_dot_stage1(const BatchSeg* __restrict__ segs, const double* __restrict__ hbase,
                                   int64_t hstride, int hoff, const double* __restrict__ x, double* w, const double* y,
                                   double* __restrict__ partials) {
  __shared__ double sbuf[256];
  const int m = blockIdx.y;
  const int64_t n = segs[m].g.ndofs, off = segs[m].off;
  const double a = hoff >= 0 ? -hbase[segs[m].member * hstride + hoff] : 0.0;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kBtDotBlocks * 256) {
    double wi = w[off + i];
    if (hoff >= 0) {
      wi = fma(a, x[off + i], wi);
      w[off + i] = wi;
    }
    acc = fma(wi, y == w ? wi : y[off + i], acc);
  }
  sbuf[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sbuf[threadIdx.x] += sbuf[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[m * kBtDotBlocks + blockIdx.x] = sbuf[0];
}
// Per member, the sum of its partials in bt_dot_stage2's order into
// out[b * ostride + ooff]; mode 1 (a norm): out = sqrt(sum), inv[b] = 1 / out (1 if 0),
// and g[b * gstride] = out if g is given; mode 2 (Arnoldi breakdown test): inv[b] = 0
// where out <= rel |out[b * ostride + doff]| + abs.
__global__ void bt_dot_stage2_to(const BatchSeg* __restrict__ segs, const double* __restrict__ partials,
                                 double* __restrict__ out, int64_t ostride, int ooff, int mode,
                                 double* __restrict__ inv, int doff, double rel, double abs_, double* __restrict__ g,
                                 int64_t gstride) {
  __shared__ double sbuf[64];
  const int m = blockIdx.x;
  sbuf[threadIdx.x] = partials[m * kBtDotBlocks + threadIdx.x];
  __syncthreads();
  for (int st = 32; st > 0; st >>= 1) {
    if (threadIdx.x < st) sbuf[threadIdx.x] += sbuf[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const int64_t b = segs[m].member;
  if (mode == 0) {
    out[b * ostride + ooff] = sbuf[0];
    return;
  }
  const double hn = sqrt(sbuf[0]);
  out[b * ostride + ooff] = hn;
  if (mode == 1) inv[b] = hn != 0.0 ? 1.0 / hn : 1.0;
  else inv[b] = hn > rel * fabs(out[b * ostride + doff]) + abs_ ? 1.0 / hn : 0.0;
  if (g) g[b * gstride] = hn;
}
// y = a_b x per member, a member-indexed
__global__ void bt_scale_dev_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs,
                                    const double* __restrict__ a, const double* x, double* y) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const int64_t i = segs[m].off + (u - segs[m].u_dof);
  y[i] = x[i] * a[segs[m].member];
}
// The FGMRES rotations of column j, one thread per member (givens_kernel's steps);
// status[seg] = the member's new residual estimate.
__global__ void bt_givens_kernel(const BatchSeg* __restrict__ segs, int nseg, double* __restrict__ Hb,
                                 double* __restrict__ csb, double* __restrict__ snb, double* __restrict__ gb, int R,
                                 int j, double* __restrict__ status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nseg) return;
  const int64_t b = segs[e].member;
  double* H = Hb + b * (int64_t)(R + 1) * R;
  double *cs = csb + b * R, *sn = snb + b * R, *g = gb + b * (R + 1);
  for (int i = 0; i < j; ++i) {
    const double hi = H[i * R + j], hi1 = H[(i + 1) * R + j];
    H[i * R + j] = cs[i] * hi + sn[i] * hi1;
    H[(i + 1) * R + j] = -sn[i] * hi + cs[i] * hi1;
  }
  const double a = H[j * R + j], c = H[(j + 1) * R + j];
  const double den = hypot(a, c);
  cs[j] = a / den;
  sn[j] = c / den;
  H[j * R + j] = den;
  H[(j + 1) * R + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  status[e] = g[j + 1];
}
// y_b = R_b^{-1} g_b (leading jend x jend triangle), one thread per member
__global__ void bt_trisolve_kernel(const BatchSeg* __restrict__ segs, int nseg, const double* __restrict__ Hb,
                                   const double* __restrict__ gb, double* __restrict__ yb, int R, int jend) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nseg) return;
  const int64_t b = segs[e].member;
  const double* H = Hb + b * (int64_t)(R + 1) * R;
  const double* g = gb + b * (R + 1);
  double* y = yb + b * R;
  for (int i = jend - 1; i >= 0; --i) {
    double acc = g[i];
    for (int l = i + 1; l < jend; ++l) acc -= H[i * R + l] * y[l];
    y[i] = acc / H[i * R + i];
  }
}
// x += sum_{l < jend} y_{b,l} Z_l per member, the terms added one after another
__global__ void bt_multi_axpy_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs,
                                     const double* __restrict__ yb, int R, KrylovBasis z, int jend,
                                     double* __restrict__ x) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const int64_t i = segs[m].off + (u - segs[m].u_dof);
  const double* y = yb + (int64_t)segs[m].member * R;
  double xi = x[i];
  for (int l = 0; l < jend; ++l) xi = fma(y[l], z.p[l][i], xi);
  x[i] = xi;
}

inline unsigned grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 4 * 152 * 8 ? (b > 0 ? b : 1) : 4 * 152 * 8);
}

}  // namespace

// shared memory of the tiled transfers (the velocity field, degree k+1, is the larger)
static size_t restrict_smem(int k) {
  const int P = k + 1, W = 2 * kTrBX + 4 * P + 1, H = 2 * kTrBY + 4 * P + 1;
  return sizeof(double) * (size_t)(H * W + H * kTrBX);
}
static size_t prolong_smem(int k) {
  const int P = k + 1, W = kTpBX / 2 + 2 * P + 1, H = kTpBY / 2 + 2 * P + 1;
  return sizeof(double) * (size_t)(H * W + H * kTpBX);
}

void launch_restrict(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xf, double* xc,
                     cudaStream_t s) {
  const dim3 grid((gc.nv + kTrBX - 1) / kTrBX, (gc.nv + kTrBY - 1) / kTrBY, (unsigned)(3 * gf.N * gf.nt));
  const size_t smem = restrict_smem(gf.k);
  if (gf.k == 1) restrict_tiled_kernel<1><<<grid, 256, smem, s>>>(gf, gc, T, xf, xc);
  else if (gf.k == 2) restrict_tiled_kernel<2><<<grid, 256, smem, s>>>(gf, gc, T, xf, xc);
  else restrict_kernel<<<(unsigned)((gc.ndofs + 255) / 256), 256, 0, s>>>(gf, gc, T, xf, xc);
  WR_LAUNCH_CHECK();
}
void launch_prolong_add(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xc, double* xf,
                        cudaStream_t s) {
  const dim3 grid((gf.nv + kTpBX - 1) / kTpBX, (gf.nv + kTpBY - 1) / kTpBY, (unsigned)(3 * gf.N * gf.nt));
  const size_t smem = prolong_smem(gf.k);
  if (gf.k == 1) prolong_tiled_kernel<1><<<grid, 256, smem, s>>>(gf, gc, T, xc, xf);
  else if (gf.k == 2) prolong_tiled_kernel<2><<<grid, 256, smem, s>>>(gf, gc, T, xc, xf);
  else prolong_add_kernel<<<(unsigned)((gf.ndofs + 255) / 256), 256, 0, s>>>(gf, gc, T, xc, xf);
  WR_LAUNCH_CHECK();
}
void launch_project_pressure(const LevelGeom& g, const FeTables& T, double* x, cudaStream_t s) {
  project_pressure_kernel<<<g.N * g.nt, 256, 0, s>>>(g, T, x);
  WR_LAUNCH_CHECK();
}
void launch_zero_dirichlet(const LevelGeom& g, double* x, cudaStream_t s) {
  zero_dirichlet_kernel<<<(unsigned)((g.ndofs + 255) / 256), 256, 0, s>>>(g, x);
  WR_LAUNCH_CHECK();
}
void launch_splitmix_free(const LevelGeom& g, uint64_t seed, double* x, cudaStream_t s) {
  splitmix_kernel<<<(unsigned)((g.ndofs + 255) / 256), 256, 0, s>>>(g, seed, x);
  WR_LAUNCH_CHECK();
}
void vec_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s) {
  axpby_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y);
  WR_LAUNCH_CHECK();
}
void vec_axpbypz(int64_t n, double a, const double* x, double b, const double* y, double c, double* z,
                 cudaStream_t s) {
  axpbypz_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y, c, z);
  WR_LAUNCH_CHECK();
}
void vec_copy(int64_t n, const double* x, double* y, cudaStream_t s) {
  copy_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, x, y);
  WR_LAUNCH_CHECK();
}
void vec_scale(int64_t n, double a, double* x, cudaStream_t s) {
  scale_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, x);
  WR_LAUNCH_CHECK();
}
void vec_zero(int64_t n, double* x, cudaStream_t s) { WR_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s)); }
int dot_partials_size() { return kDotBlocks; }
void vec_dot_dev(int64_t n, const double* x, const double* y, double* partials, double* out, cudaStream_t s) {
  dot_stage1<<<kDotBlocks, kDotThreads, 0, s>>>(n, x, y, partials);
  WR_LAUNCH_CHECK();
  dot_stage2<<<1, kDotThreads, 0, s>>>(partials, out);
  WR_LAUNCH_CHECK();
}

void krylov_axpy_dot(int64_t n, const double* h, const double* x, double* w, const double* y, double* partials,
                     unsigned* count, double* out, cudaStream_t s) {
  axpy_dot_kernel<<<krylov_blocks(n), kDotThreads, 0, s>>>(n, h, x, w, y, partials, count, out, 0, nullptr, nullptr,
                                                          0.0, 0.0);
  WR_LAUNCH_CHECK();
}
void krylov_axpy_norm(int64_t n, const double* h, const double* x, double* w, double* partials, unsigned* count,
                      double* out, double* inv, const double* diag, double rel, double abs_, cudaStream_t s) {
  axpy_dot_kernel<<<krylov_blocks(n), kDotThreads, 0, s>>>(n, h, x, w, w, partials, count, out, diag ? 2 : 1, inv,
                                                          diag, rel, abs_);
  WR_LAUNCH_CHECK();
}
int64_t mgs_small_limit() { return 8192; }
void krylov_mgs_small(int64_t n, const KrylovBasis& V, int j, double* w, double* H, int m, int col, bool breakdown,
                      cudaStream_t s) {
  mgs_small_kernel<<<1, kMgsThreads, 0, s>>>(n, V, j, w, H, m, col, breakdown ? 2 : 1, 1e-14, 1e-300);
  WR_LAUNCH_CHECK();
}
void vec_scale_dev(int64_t n, const double* a, const double* x, double* y, cudaStream_t s) {
  scale_dev_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, y);
  WR_LAUNCH_CHECK();
}
void krylov_givens(double* H, double* cs, double* sn, double* g, int j, int m, double* status, cudaStream_t s) {
  givens_kernel<<<1, 1, 0, s>>>(H, cs, sn, g, j, m, status);
  WR_LAUNCH_CHECK();
}
void krylov_update(int64_t n, const double* H, const double* g, double* y, int jend, int m, const KrylovBasis& z,
                   double* x, cudaStream_t s) {
  if (jend <= 0) return;
  trisolve_kernel<<<1, 1, 0, s>>>(H, g, y, jend, m);
  WR_LAUNCH_CHECK();
  multi_axpy_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, y, z, jend, x);
  WR_LAUNCH_CHECK();
}

double measure_fp64_tflops(cudaStream_t s) {
  int dev = 0, sms = 0;
  WR_CUDA(cudaGetDevice(&dev));
  WR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 13;
  double* out = nullptr;
  WR_CUDA(cudaMalloc(&out, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  WR_CUDA(cudaEventCreate(&e0));
  WR_CUDA(cudaEventCreate(&e1));
  fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
  WR_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < 5; ++r) fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
  WR_CUDA(cudaEventRecord(e1, s));
  WR_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  WR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 5.0 * blocks * threads * (double)iters * 8 * 2;
  return flops / (ms * 1e-3) / 1e12;
}

static unsigned nblocks(int64_t n) { return (unsigned)((n + 255) / 256); }

void bt_restrict(const BatchSeg* segs, int nseg, int64_t dofsc, const FeTables& T, const double* xf, double* xc,
                 cudaStream_t s) {
  if (dofsc <= 0) return;
  bt_restrict_kernel<<<nblocks(dofsc), 256, 0, s>>>(segs, nseg, dofsc, T, xf, xc);
  WR_LAUNCH_CHECK();
}
void bt_prolong_add(const BatchSeg* segs, int nseg, int64_t dofs, const FeTables& T, const double* xc, double* xf,
                    cudaStream_t s) {
  if (dofs <= 0) return;
  bt_prolong_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, T, xc, xf);
  WR_LAUNCH_CHECK();
}
void bt_project_pressure(const BatchSeg* segs, int nseg, int64_t tblks, const FeTables& T, double* x, bool absolute,
                         cudaStream_t s) {
  if (tblks <= 0) return;
  bt_project_kernel<<<(unsigned)tblks, 256, 0, s>>>(segs, nseg, T, x, absolute ? 1 : 0);
  WR_LAUNCH_CHECK();
}
void bt_splitmix(const BatchSeg* segs, int nseg, int64_t dofs, const int64_t* seeds, double* x, cudaStream_t s) {
  if (dofs <= 0) return;
  bt_splitmix_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, seeds, x);
  WR_LAUNCH_CHECK();
}
void bt_axpby(const BatchSeg* segs, int nseg, int64_t dofs, const double* a, double as, const double* x,
              const double* b, double bs_, double* y, cudaStream_t s) {
  if (dofs <= 0) return;
  bt_axpby_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, a, as, x, b, bs_, y);
  WR_LAUNCH_CHECK();
}
void bt_copy(const BatchSeg* segs, int nseg, int64_t dofs, const double* x, double* y, cudaStream_t s) {
  if (dofs <= 0) return;
  bt_copy_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, x, y);
  WR_LAUNCH_CHECK();
}
void bt_fill_abs(const BatchSeg* segs, int nseg, int64_t dofs, double v, cudaStream_t s) {
  if (dofs <= 0) return;
  bt_fill_abs_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, v);
  WR_LAUNCH_CHECK();
}
int bt_dot_blocks() { return kBtDotBlocks; }
void bt_dot(const BatchSeg* segs, int nseg, const double* x, const double* y, double* partials, double* out,
            cudaStream_t s) {
  if (nseg <= 0) return;
  bt_dot_stage1<<<dim3(kBtDotBlocks, nseg), 256, 0, s>>>(segs, x, y, partials);
  WR_LAUNCH_CHECK();
  bt_dot_stage2<<<nseg, kBtDotBlocks, 0, s>>>(partials, out);
  WR_LAUNCH_CHECK();
}

void bt_axpy_dot(const BatchSeg* segs, int nseg, const double* hbase, int64_t hstride, int hoff, const double* x,
                 double* w, const double* y, double* partials, double* out, int64_t ostride, int ooff,
                 cudaStream_t s) {
  if (!nseg) return;
  bt_axpy_dot_stage1<<<dim3(kBtDotBlocks, nseg), 256, 0, s>>>(segs, hbase, hstride, hoff, x, w, y, partials);
  WR_LAUNCH_CHECK();
  bt_dot_stage2_to<<<nseg, kBtDotBlocks, 0, s>>>(segs, partials, out, ostride, ooff, 0, nullptr, 0, 0.0, 0.0, nullptr,
                                                 0);
  WR_LAUNCH_CHECK();
}
void bt_axpy_norm(const BatchSeg* segs, int nseg, const double* hbase, int64_t hstride, int hoff, const double* x,
                  double* w, double* partials, double* out, int64_t ostride, int ooff, double* inv, int doff,
                  double* g, int64_t gstride, cudaStream_t s) {
  if (!nseg) return;
  bt_axpy_dot_stage1<<<dim3(kBtDotBlocks, nseg), 256, 0, s>>>(segs, hbase, hstride, hoff, x, w, w, partials);
  WR_LAUNCH_CHECK();
  bt_dot_stage2_to<<<nseg, kBtDotBlocks, 0, s>>>(segs, partials, out, ostride, ooff, doff >= 0 ? 2 : 1, inv, doff,
                                                 1e-14, 1e-300, g, gstride);
  WR_LAUNCH_CHECK();
}
void bt_scale_dev(const BatchSeg* segs, int nseg, int64_t dofs, const double* a, const double* x, double* y,
                  cudaStream_t s) {
  if (!nseg || !dofs) return;
  bt_scale_dev_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, a, x, y);
  WR_LAUNCH_CHECK();
}
void bt_givens(const BatchSeg* segs, int nseg, double* H, double* cs, double* sn, double* g, int R, int j,
               double* status, cudaStream_t s) {
  if (!nseg) return;
  bt_givens_kernel<<<(nseg + 127) / 128, 128, 0, s>>>(segs, nseg, H, cs, sn, g, R, j, status);
  WR_LAUNCH_CHECK();
}
void bt_krylov_update(const BatchSeg* segs, int nseg, int64_t dofs, const double* H, const double* g, double* y, int R,
                      int jend, const KrylovBasis& z, double* x, cudaStream_t s) {
  if (!nseg || jend <= 0) return;
  bt_trisolve_kernel<<<(nseg + 127) / 128, 128, 0, s>>>(segs, nseg, H, g, y, R, jend);
  WR_LAUNCH_CHECK();
  bt_multi_axpy_kernel<<<nblocks(dofs), 256, 0, s>>>(segs, nseg, dofs, y, R, z, jend, x);
  WR_LAUNCH_CHECK();
}
