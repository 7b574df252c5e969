// Heat-equation waveform relaxation on the GPU (Def. heat, Sec. 3, Sec. 5).
//
// u_t - nu lap u = 0 with natural boundary conditions, DG(q) in time (q = 0..3,
// right-Radau Lagrange basis), continuous Q_k (k = 1, 2, 3) on an n x n mesh (the
// degrees of the paper's heat experiments, Sec. 5).  One scalar
// field per temporal DoF: the canonical index is (slab (q+1) + a) S + y nv + x with
// nv = n k + 1, S = nv^2.  Every operator is a tensor product of global 1D
// matrices on the Cartesian mesh:
//   J:  rows (n, a):  sum_b Kt[a,b] M u_{n,b} + dt nu Wt[a,b] K u_{n,b} - tau_a(0) M u_{n-1,q},
//   M = M1 (x) M1,  K = K1 (x) M1 + M1 (x) K1,
// applied matrix-free, one output DoF per thread.  The vertex-star patch of
// vertex (I, J) holds the nodes of its open star, a (2k-1)^2 window starting at
// node ((I-1)k+1, (J-1)k+1) (clipped to the domain); its slab blocks are the
// principal submatrices of J, inverted per (patch, slab) and applied by forward
// substitution over slabs.  The coarsest level (2x2 cells, or 1x1 where the 2x2
// block would not fit in shared memory) is one block holding every node.  Levels coarsen in space only; transfers are the tensor products of
// the 1D degree-k Lagrange interpolation.
#include "wrmg_internal.h"

namespace {

// global 1D entry of a degree-P Lagrange matrix: sum over the cells holding both nodes
template <int P>
__device__ __forceinline__ double heat_1d(const double (*ref)[WR_MAX_NVL], int n, int gi, int gj) {
  const int lo0 = gi == 0 ? 0 : (gi - 1) / P, lo1 = gj == 0 ? 0 : (gj - 1) / P;
  const int hi0 = min(gi / P, n - 1), hi1 = min(gj / P, n - 1);
  double v = 0.0;
  for (int c = max(lo0, lo1); c <= min(hi0, hi1); ++c) v += ref[gi - P * c][gj - P * c];
  return v;
}

__device__ __forceinline__ double heat_initial(const PhysParams& ph, double x, double y) {
  if (ph.kind == WR_HEAT_EIGEN) return cospi(x);
  return sinpi(x) + cospi(2.0 * y);
}

// The reference tables the heat kernels index with thread-dependent indices, copied
// once per CTA into shared memory (kernel-parameter space serves one address at a time).
struct HeatTab {
  double m1[WR_MAX_NVL][WR_MAX_NVL], k1[WR_MAX_NVL][WR_MAX_NVL];
  double Kt[WR_MAX_NT][WR_MAX_NT], Wt[WR_MAX_NT][WR_MAX_NT], tau0[WR_MAX_NT];
};

__device__ __forceinline__ void stage_heat_tab(const FeTables& T, HeatTab& t) {
  for (int e = threadIdx.x; e < WR_MAX_NVL * WR_MAX_NVL; e += blockDim.x) {
    const int i = e / WR_MAX_NVL, j = e % WR_MAX_NVL;
    t.m1[i][j] = T.m1[i][j];
    t.k1[i][j] = T.k1[i][j];
  }
  for (int e = threadIdx.x; e < WR_MAX_NT * WR_MAX_NT; e += blockDim.x) {
    const int a = e / WR_MAX_NT, b = e % WR_MAX_NT;
    t.Kt[a][b] = T.Kt[a][b];
    t.Wt[a][b] = T.Wt[a][b];
  }
  for (int a = threadIdx.x; a < WR_MAX_NT; a += blockDim.x) t.tau0[a] = T.tau0[a];
}

// y = J x (RES = false) or F(x) = J x - b (RES = true: the slab-0 initial-data term),
// by tensor-product passes.  On slab n,
//   y_a = sum_b Kt[a][b] M x_b + dt nu sum_b Wt[a][b] K x_b - tau_a(0) M x^-,
// M = My (x) Mx, K = Ky (x) Mx + My (x) Kx (global 1D matrices with 2K+1 bands), x^- the
// last temporal DoF of slab n-1 (slab 0: the initial data for F, zero for J).
// Pass 1 (x direction), one thread per (slab, component, node), components
// x_0 .. x_{NT-1} and x^-:  tM = Mx x_c and tK = Kx x_c along each mesh row, stored
// [slab][c][tM, tK][node].  Pass 2 (y direction and the temporal mixing), one thread
// per (slab, node): M x_b = My tM_b, K x_b = Ky tM_b + My tK_b, M x^- = My tM_NT, then
// every a.  About 50 FP64 operations per DoF instead of a (2K+1)^2-tap stencil with
// its coefficients formed per tap.
template <int K, int Q, bool RES>
__global__ void heat_xpass_kernel(LevelGeom g, FeTables Tp, PhysParams ph, const double* __restrict__ x,
                                  double* __restrict__ t) {
  constexpr int NT = Q + 1, NC = NT + 1;
  __shared__ HeatTab T;
  stage_heat_tab(Tp, T);
  __syncthreads();
  const int S = g.S, nv = g.nv;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.N * NC * S) return;
  const int sp = int(idx % S);
  const int64_t sc = idx / S;
  const int c = int(sc % NC), slab = int(sc / NC);
  const int ix = sp % nv, iy = sp / nv;
  const double h = g.h, ih = 1.0 / h;
  double am = 0.0, ak = 0.0;
#pragma unroll
  for (int d = 0; d <= 2 * K; ++d) {
    const int jx = ix - K + d;
    if (jx < 0 || jx >= nv) continue;
    const int64_t node = (int64_t)iy * nv + jx;
    double v;
    if (c < NT) {
      v = x[((int64_t)slab * NT + c) * S + node];
    } else if (slab > 0) {
      v = x[((int64_t)(slab - 1) * NT + NT - 1) * S + node];
    } else if (RES) {
      v = ph.u0 ? ph.u0[node] : heat_initial(ph, jx * (h / K), iy * (h / K));
    } else {
      v = 0.0;
    }
    am = fma(h * heat_1d<K>(T.m1, g.n, ix, jx), v, am);
    ak = fma(ih * heat_1d<K>(T.k1, g.n, ix, jx), v, ak);
  }
  double* tc = t + (sc * 2) * S;
  tc[sp] = am;
  tc[S + sp] = ak;
}

template <int K, int Q>
__global__ void heat_ypass_kernel(LevelGeom g, FeTables Tp, PhysParams ph, const double* __restrict__ t,
                                  double* __restrict__ y) {
  constexpr int NT = Q + 1, NC = NT + 1;
  __shared__ HeatTab T;
  stage_heat_tab(Tp, T);
  __syncthreads();
  const int S = g.S, nv = g.nv;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.N * S) return;
  const int sp = int(idx % S), slab = int(idx / S);
  const int ix = sp % nv, iy = sp / nv;
  const double h = g.h, ih = 1.0 / h, cdt = g.dt * ph.nu;
  double my[2 * K + 1], ky[2 * K + 1];
#pragma unroll
  for (int d = 0; d <= 2 * K; ++d) {
    const int jy = iy - K + d;
    const bool ok = jy >= 0 && jy < nv;
    my[d] = ok ? h * heat_1d<K>(T.m1, g.n, iy, jy) : 0.0;
    ky[d] = ok ? ih * heat_1d<K>(T.k1, g.n, iy, jy) : 0.0;
  }
  double Mb[NT], Kb[NT], Mp = 0.0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double* tc = t + (((int64_t)slab * NC + c) * 2) * S;
    double m = 0.0, kk = 0.0;
#pragma unroll
    for (int d = 0; d <= 2 * K; ++d) {
      const int jy = iy - K + d;
      if (jy < 0 || jy >= nv) continue;
      const int64_t node = (int64_t)jy * nv + ix;
      const double tm = tc[node];
      m = fma(my[d], tm, m);
      if (c < NT) kk = fma(ky[d], tm, fma(my[d], tc[S + node], kk));
    }
    if (c < NT) {
      Mb[c] = m;
      Kb[c] = kk;
    } else {
      Mp = m;
    }
  }
#pragma unroll
  for (int a = 0; a < NT; ++a) {
    double acc = -T.tau0[a] * Mp;
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      acc = fma(T.Kt[a][b], Mb[b], acc);
      acc = fma(cdt * T.Wt[a][b], Kb[b], acc);
    }
    y[((int64_t)slab * NT + a) * S + sp] = acc;
  }
}

// Block layout: PX x PX node window per temporal DoF, slot = a PX^2 + ly PX + lx;
// slots outside the domain are padding (identity rows and columns).  WHOLE: the
// block of the coarsest level (PX = n k + 1, every node); else a vertex-star patch.
template <int K, int PX, bool WHOLE>
struct HeatBlock {
  __device__ static void origin(const LevelGeom& g, int blk, int& x0, int& y0) {
    if (!WHOLE) {  // vertex-star patch
      const int I = blk % (g.n + 1), J = blk / (g.n + 1);
      x0 = (I - 1) * K + 1;
      y0 = (J - 1) * K + 1;
    } else {  // the whole coarsest mesh
      x0 = y0 = 0;
    }
  }
};

// Inverts the slab block of (block, slab): assembled in shared memory, Gauss-Jordan
// with partial pivoting (largest |.|, lowest row on ties), stored column-major.
template <int K, int Q, int PX, bool WHOLE, int NTH>
__global__ void __launch_bounds__(NTH) heat_factor_kernel(LevelGeom g, FeTables Tp, PhysParams ph,
                                                          double* __restrict__ factors, int* __restrict__ status) {
  constexpr int NT = Q + 1, P2 = PX * PX, M = NT * P2;
  extern __shared__ __align__(16) double sA[];  // M x M row-major, then one pivot column
  __shared__ int piv;
  __shared__ HeatTab T;
  stage_heat_tab(Tp, T);
  __syncthreads();
  const int blk = blockIdx.x, slab = blockIdx.y, tid = threadIdx.x;
  int x0, y0;
  HeatBlock<K, PX, WHOLE>::origin(g, blk, x0, y0);
  const int nv = g.nv;
  const double h = g.h, ih = 1.0 / h, cdt = g.dt * ph.nu;
  for (int e = tid; e < M * M; e += NTH) {
    const int i = e / M, j = e % M;
    const int a = i / P2, si = i % P2, b = j / P2, sj = j % P2;
    const int ix = x0 + si % PX, iy = y0 + si / PX, jx = x0 + sj % PX, jy = y0 + sj / PX;
    const bool vi = ix >= 0 && ix < nv && iy >= 0 && iy < nv, vj = jx >= 0 && jx < nv && jy >= 0 && jy < nv;
    double v;
    if (!vi || !vj) {
      v = (i == j) ? 1.0 : 0.0;
    } else {
      const double mxx = h * heat_1d<K>(T.m1, g.n, ix, jx), myy = h * heat_1d<K>(T.m1, g.n, iy, jy);
      const double kxx = ih * heat_1d<K>(T.k1, g.n, ix, jx), kyy = ih * heat_1d<K>(T.k1, g.n, iy, jy);
      v = T.Kt[a][b] * (myy * mxx) + cdt * T.Wt[a][b] * (kyy * mxx + myy * kxx);
    }
    sA[i * M + j] = v;
  }
  __syncthreads();
  double* col = sA + M * M;
  __shared__ int perm[M];
  __shared__ double pinv;  // the pivot's reciprocal, formed once per step
  bool singular = false;
  for (int p = 0; p < M; ++p) {
    if (tid < 32) {  // warp 0: largest |.| (compared as sign-cleared bit patterns), lowest row on ties
      unsigned long long best = 0;
      int bi = M;
      for (int i = p + tid; i < M; i += 32) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(sA[i * M + p]) & 0x7fffffffffffffffull;
        if (v > best || bi == M) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        piv = bi;
        perm[p] = bi;
        pinv = 1.0 / sA[bi * M + p];
      }
    }
    __syncthreads();
    const int r = piv;
    if (r != p)
      for (int j = tid; j < M; j += NTH) {
        const double t = sA[p * M + j];
        sA[p * M + j] = sA[r * M + j];
        sA[r * M + j] = t;
      }
    __syncthreads();
    const double d = sA[p * M + p];
    if (!(fabs(d) > 0.0)) singular = true;
    const double inv = pinv;
    for (int i = tid; i < M; i += NTH) col[i] = sA[i * M + p];
    __syncthreads();
    for (int j = tid; j < M; j += NTH) sA[p * M + j] = (j == p ? 1.0 : sA[p * M + j]) * inv;
    __syncthreads();
    for (int e = tid; e < M * M; e += NTH) {
      const int i = e / M, j = e % M;
      if (i == p) continue;
      const double f = col[i];
      sA[i * M + j] = (j == p ? 0.0 : sA[i * M + j]) - f * sA[p * M + j];
    }
    __syncthreads();
  }
  // undo the row exchanges as column exchanges of the inverse, last to first
  for (int p = M - 1; p >= 0; --p) {
    const int r = perm[p];
    if (r != p)
      for (int i = tid; i < M; i += NTH) {
        const double t = sA[i * M + p];
        sA[i * M + p] = sA[i * M + r];
        sA[i * M + r] = t;
      }
    __syncthreads();
  }
  double* out = factors + ((int64_t)blk * g.N + slab) * M * M;
  for (int e = tid; e < M * M; e += NTH) {
    const int j = e / M, i = e % M;  // column-major store
    out[e] = sA[i * M + j];
  }
  if (singular && tid == 0) atomicExch(status, 1);
}

// Forward substitution over slabs for one block per CTA: rhs = r_n - L y_{n-1},
// y_n = A_nn^{-1} rhs; L = -tau(0) (x) M restricted to the block's nodes.
// Patches write [slab][block][slot] outputs; the coarse block writes the solution.
template <int K, int Q, int PX, bool WHOLE, int NTH>
__global__ void __launch_bounds__(NTH) heat_apply_kernel(LevelGeom g, FeTables Tp, const double* __restrict__ factors,
                                                         const double* __restrict__ r, double* __restrict__ out,
                                                         int nblk) {
  constexpr int NT = Q + 1, P2 = PX * PX, M = NT * P2;
  __shared__ double rhs[M], yv[M], ylast[P2], tj[P2], mj[P2], m1x[PX][PX], m1y[PX][PX];
  __shared__ int node[P2];
  __shared__ HeatTab T;
  stage_heat_tab(Tp, T);
  __syncthreads();
  const int blk = blockIdx.x, tid = threadIdx.x;
  int x0, y0;
  HeatBlock<K, PX, WHOLE>::origin(g, blk, x0, y0);
  const int nv = g.nv;
  for (int s = tid; s < P2; s += NTH) {
    const int ix = x0 + s % PX, iy = y0 + s / PX;
    node[s] = (ix >= 0 && ix < nv && iy >= 0 && iy < nv) ? iy * nv + ix : -1;
    ylast[s] = 0.0;
  }
  for (int e = tid; e < PX * PX; e += NTH) {
    const int i = e / PX, j = e % PX;
    const int xi = x0 + i, xj = x0 + j, yi = y0 + i, yj = y0 + j;
    m1x[i][j] = (xi >= 0 && xi < nv && xj >= 0 && xj < nv) ? g.h * heat_1d<K>(T.m1, g.n, xi, xj) : 0.0;
    m1y[i][j] = (yi >= 0 && yi < nv && yj >= 0 && yj < nv) ? g.h * heat_1d<K>(T.m1, g.n, yi, yj) : 0.0;
  }
  __syncthreads();
  for (int slab = 0; slab < g.N; ++slab) {
    if (slab > 0) {  // jump term M y_{n-1, last} on the block's nodes, one tensor direction at a time
      for (int e = tid; e < P2; e += NTH) {
        const int ly = e / PX, jx = e % PX;
        double t = 0.0;
        for (int jy = 0; jy < PX; ++jy) t = fma(m1y[ly][jy], ylast[jy * PX + jx], t);
        tj[e] = t;
      }
      __syncthreads();
      for (int e = tid; e < P2; e += NTH) {
        const int ly = e / PX, lx = e % PX;
        double m = 0.0;
        for (int jx = 0; jx < PX; ++jx) m = fma(m1x[lx][jx], tj[ly * PX + jx], m);
        mj[e] = m;
      }
      __syncthreads();
    }
    for (int i = tid; i < M; i += NTH) {
      const int a = i / P2, si = i % P2, nd = node[si];
      double v = nd >= 0 ? r[((int64_t)slab * NT + a) * g.S + nd] : 0.0;
      if (slab > 0 && nd >= 0) v = fma(T.tau0[a], mj[si], v);
      rhs[i] = v;
    }
    __syncthreads();
    const double* A = factors + ((int64_t)blk * g.N + slab) * M * M;
    for (int i = tid; i < M; i += NTH) {
      double acc = 0.0;
      for (int j = 0; j < M; ++j) acc = fma(A[(int64_t)j * M + i], rhs[j], acc);
      yv[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < M; i += NTH) {
      const int a = i / P2, si = i % P2;
      if (!WHOLE) {
        out[((int64_t)slab * nblk + blk) * M + i] = yv[i];
      } else if (node[si] >= 0) {
        out[((int64_t)slab * NT + a) * g.S + node[si]] = yv[i];
      }
      if (a == NT - 1) ylast[si] = yv[i];
    }
    __syncthreads();
  }
}

// y = sum over the patches holding each node of their outputs (pull, fixed order).
template <int K, int Q>
__global__ void heat_scatter_kernel(LevelGeom g, const double* __restrict__ Yp, double* __restrict__ y) {
  constexpr int NT = Q + 1, PX = 2 * K - 1, P2 = PX * PX, M = NT * P2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  const int nv = g.nv, n1 = g.n + 1;
  const int64_t blk = idx / g.S;
  const int sp = int(idx % g.S), slab = int(blk / NT), a = int(blk % NT);
  const int gx = sp % nv, gy = sp / nv;
  const int Ix0 = gx % K == 0 ? gx / K : gx / K, Ix1 = gx % K == 0 ? gx / K : min(gx / K + 1, g.n);
  const int Iy0 = gy % K == 0 ? gy / K : gy / K, Iy1 = gy % K == 0 ? gy / K : min(gy / K + 1, g.n);
  double acc = 0.0;
  for (int J = Iy0; J <= Iy1; ++J)
    for (int I = Ix0; I <= Ix1; ++I) {
      const int lx = gx - ((I - 1) * K + 1), ly = gy - ((J - 1) * K + 1);
      acc += Yp[((int64_t)slab * n1 * n1 + J * n1 + I) * M + a * P2 + ly * PX + lx];
    }
  y[idx] = acc;
}

// prolongation weight of coarse node c at fine node f (degree-K 1D Lagrange interpolation)
template <int K>
__device__ __forceinline__ double heat_p1(const FeTables& T, int nc, int f, int c) {
  int cell = f / (2 * K);
  if (cell > nc - 1) cell = nc - 1;
  const int rr = f - 2 * K * cell, l = c - K * cell;
  return (l >= 0 && l <= K) ? T.pv[rr][l] : 0.0;
}

// xf += P xc (pull over the coarse nodes of each fine node's coarse cell)
template <int K>
__global__ void heat_prolong_kernel(LevelGeom gf, LevelGeom gc, FeTables T, const double* __restrict__ xc,
                                    double* __restrict__ xf) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= gf.ndofs) return;
  const int64_t blk = idx / gf.S;
  const int sp = int(idx % gf.S), fx = sp % gf.nv, fy = sp / gf.nv;
  const int cxc = min(fx / (2 * K), gc.n - 1), cyc = min(fy / (2 * K), gc.n - 1);
  double acc = 0.0;
  for (int ly = 0; ly <= K; ++ly) {
    const int cy = cyc * K + ly;
    const double wy = heat_p1<K>(T, gc.n, fy, cy);
    if (wy == 0.0) continue;
    for (int lx = 0; lx <= K; ++lx) {
      const int cx = cxc * K + lx;
      const double wx = heat_p1<K>(T, gc.n, fx, cx);
      if (wx != 0.0) acc = fma(wy * wx, xc[blk * gc.S + (int64_t)cy * gc.nv + cx], acc);
    }
  }
  xf[idx] += acc;
}

// xc = P^T xf (pull over the fine nodes whose coarse cell holds the coarse node)
template <int K>
__global__ void heat_restrict_kernel(LevelGeom gf, LevelGeom gc, FeTables T, const double* __restrict__ xf,
                                     double* __restrict__ xc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= gc.ndofs) return;
  const int64_t blk = idx / gc.S;
  const int sp = int(idx % gc.S), cx = sp % gc.nv, cy = sp / gc.nv;
  const int fx0 = max(0, 2 * (cx - K)), fx1 = min(gf.nv - 1, 2 * (cx + K));
  const int fy0 = max(0, 2 * (cy - K)), fy1 = min(gf.nv - 1, 2 * (cy + K));
  double acc = 0.0;
  for (int fy = fy0; fy <= fy1; ++fy) {
    const double wy = heat_p1<K>(T, gc.n, fy, cy);
    if (wy == 0.0) continue;
    for (int fx = fx0; fx <= fx1; ++fx) {
      const double wx = heat_p1<K>(T, gc.n, fx, cx);
      if (wx != 0.0) acc = fma(wy * wx, xf[blk * gf.S + (int64_t)fy * gf.nv + fx], acc);
    }
  }
  xc[idx] = acc;
}

// uniform(-1, 1) on every DoF, the splitmix64 generator of the Navier-Stokes path
__global__ void heat_splitmix_kernel(int64_t n, uint64_t seed, double* __restrict__ x) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  uint64_t z = seed + (uint64_t)(idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  x[idx] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// node index (or -1 outside the domain) of every slot of one patch, from the kernels' own layout
template <int K>
__global__ void heat_patch_slots_kernel(LevelGeom g, int blk, int* __restrict__ out) {
  constexpr int PX = 2 * K - 1;
  const int s = threadIdx.x;
  if (s >= PX * PX) return;
  int x0, y0;
  HeatBlock<K, PX, false>::origin(g, blk, x0, y0);
  const int ix = x0 + s % PX, iy = y0 + s / PX;
  out[s] = (ix >= 0 && ix < g.nv && iy >= 0 && iy < g.nv) ? iy * g.nv + ix : -1;
}

unsigned grid_of(int64_t n) { return (unsigned)((n + 255) / 256); }

// The factor kernel holds one M x M FP64 block (+ a column) in shared memory.
constexpr size_t kHeatSmemLimit = 227 * 1024;
constexpr size_t heat_factor_smem(int m) { return sizeof(double) * ((size_t)m * m + m); }
constexpr int heat_threads(int m) { return m <= 32 ? 32 : (m <= 64 ? 64 : (m <= 128 ? 128 : 256)); }

template <int K, int Q, int PX, bool WHOLE>
void run_heat_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph, int nblk, double* f, int* st,
                     cudaStream_t s) {
  constexpr int M = (Q + 1) * PX * PX, NTH = heat_threads(M);
  if constexpr (heat_factor_smem(M) > kHeatSmemLimit) {
    throw WrError(WR_ERR_ARG, "heat: the coarse block does not fit in shared memory (use a 1x1 coarsest mesh)");
  } else {
    const size_t smem = heat_factor_smem(M);
    auto kern = heat_factor_kernel<K, Q, PX, WHOLE, NTH>;
    WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3(nblk, g.N), NTH, smem, s>>>(g, T, ph, f, st);
    WR_LAUNCH_CHECK();
  }
}

template <int K, int Q, int PX, bool WHOLE>
void run_heat_apply(const LevelGeom& g, const FeTables& T, const double* f, const double* r, double* out, int nblk,
                    cudaStream_t s) {
  constexpr int M = (Q + 1) * PX * PX, NTH = heat_threads(M);
  if constexpr (heat_factor_smem(M) > kHeatSmemLimit) {
    throw WrError(WR_ERR_ARG, "heat: the coarse block does not fit in shared memory (use a 1x1 coarsest mesh)");
  } else {
    heat_apply_kernel<K, Q, PX, WHOLE, NTH><<<nblk, NTH, 0, s>>>(g, T, f, r, out, nblk);
    WR_LAUNCH_CHECK();
  }
}

}  // namespace

LevelGeom make_heat_geom(int n, int k, int q, int N, double T) {
  LevelGeom g;
  g.n = n; g.k = k; g.q = q; g.N = N; g.nt = q + 1;
  g.nv = n * k + 1;
  g.np = 0;
  g.S = g.nv * g.nv;
  g.ndofs = (int64_t)N * g.nt * g.S;
  g.h = 1.0 / n;
  g.dt = T / N;
  return g;
}

int heat_block_size(int k, int q, int n_whole) {
  const int px = n_whole > 0 ? n_whole * k + 1 : 2 * k - 1;
  return (q + 1) * px * px;
}

bool heat_block_fits(int k, int q, int n_whole) { return heat_factor_smem(heat_block_size(k, q, n_whole)) <= kHeatSmemLimit; }

#define HEAT_KQ(stmt)                                                       \
  if (g.k == 1 && g.q == 0) { constexpr int K = 1, Q = 0; stmt; }           \
  else if (g.k == 1 && g.q == 1) { constexpr int K = 1, Q = 1; stmt; }      \
  else if (g.k == 2 && g.q == 0) { constexpr int K = 2, Q = 0; stmt; }      \
  else if (g.k == 2 && g.q == 1) { constexpr int K = 2, Q = 1; stmt; }      \
  else if (g.k == 3 && g.q == 0) { constexpr int K = 3, Q = 0; stmt; }      \
  else if (g.k == 3 && g.q == 1) { constexpr int K = 3, Q = 1; stmt; }      \
  else if (g.k == 1 && g.q == 2) { constexpr int K = 1, Q = 2; stmt; }      \
  else if (g.k == 1 && g.q == 3) { constexpr int K = 1, Q = 3; stmt; }      \
  else if (g.k == 2 && g.q == 2) { constexpr int K = 2, Q = 2; stmt; }      \
  else if (g.k == 2 && g.q == 3) { constexpr int K = 2, Q = 3; stmt; }      \
  else if (g.k == 3 && g.q == 2) { constexpr int K = 3, Q = 2; stmt; }      \
  else if (g.k == 3 && g.q == 3) { constexpr int K = 3, Q = 3; stmt; }      \
  else throw WrError(WR_ERR_ARG, "heat: k must be 1..3 and q 0..3");

size_t heat_op_scratch(const LevelGeom& g) { return (size_t)g.N * (g.nt + 1) * 2 * g.S; }

void heat_jacobian(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* x, double* y,
                   double* tmp, cudaStream_t s) {
  const int64_t n1 = (int64_t)g.N * (g.nt + 1) * g.S, n2 = (int64_t)g.N * g.S;
  HEAT_KQ((heat_xpass_kernel<K, Q, false><<<grid_of(n1), 256, 0, s>>>(g, T, ph, x, tmp)));
  WR_LAUNCH_CHECK();
  HEAT_KQ((heat_ypass_kernel<K, Q><<<grid_of(n2), 256, 0, s>>>(g, T, ph, tmp, y)));
  WR_LAUNCH_CHECK();
}

void heat_residual(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* x, double* y,
                   double* tmp, cudaStream_t s) {
  const int64_t n1 = (int64_t)g.N * (g.nt + 1) * g.S, n2 = (int64_t)g.N * g.S;
  HEAT_KQ((heat_xpass_kernel<K, Q, true><<<grid_of(n1), 256, 0, s>>>(g, T, ph, x, tmp)));
  WR_LAUNCH_CHECK();
  HEAT_KQ((heat_ypass_kernel<K, Q><<<grid_of(n2), 256, 0, s>>>(g, T, ph, tmp, y)));
  WR_LAUNCH_CHECK();
}

void heat_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph, bool coarse, double* f, int* st,
                 cudaStream_t s) {
  WR_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
  if (coarse && g.n == 2) {
    HEAT_KQ((run_heat_factor<K, Q, 2 * K + 1, true>(g, T, ph, 1, f, st, s)));
  } else if (coarse && g.n == 1) {
    HEAT_KQ((run_heat_factor<K, Q, K + 1, true>(g, T, ph, 1, f, st, s)));
  } else if (coarse) {
    throw WrError(WR_ERR_ARG, "heat: the coarsest mesh must be 1x1 or 2x2");
  } else {
    HEAT_KQ((run_heat_factor<K, Q, 2 * K - 1, false>(g, T, ph, g.npatch(), f, st, s)));
  }
  int h = 0;
  WR_CUDA(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  WR_CUDA(cudaStreamSynchronize(s));
  if (h) throw WrError(WR_ERR_NAN, "singular heat patch block (zero pivot)");
}

void heat_patch_apply(const LevelGeom& g, const FeTables& T, const double* f, const double* r, double* Yp, double* y,
                      cudaStream_t s) {
  HEAT_KQ((run_heat_apply<K, Q, 2 * K - 1, false>(g, T, f, r, Yp, g.npatch(), s)));
  HEAT_KQ((heat_scatter_kernel<K, Q><<<grid_of(g.ndofs), 256, 0, s>>>(g, Yp, y)));
  WR_LAUNCH_CHECK();
}

void heat_coarse_apply(const LevelGeom& g, const FeTables& T, const double* f, const double* b, double* x,
                       cudaStream_t s) {
  if (g.n == 2) {
    HEAT_KQ((run_heat_apply<K, Q, 2 * K + 1, true>(g, T, f, b, x, 1, s)));
  } else if (g.n == 1) {
    HEAT_KQ((run_heat_apply<K, Q, K + 1, true>(g, T, f, b, x, 1, s)));
  } else {
    throw WrError(WR_ERR_ARG, "heat: the coarsest mesh must be 1x1 or 2x2");
  }
}

void heat_restrict(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xf, double* xc,
                   cudaStream_t s) {
  if (gf.k == 1) heat_restrict_kernel<1><<<grid_of(gc.ndofs), 256, 0, s>>>(gf, gc, T, xf, xc);
  else if (gf.k == 2) heat_restrict_kernel<2><<<grid_of(gc.ndofs), 256, 0, s>>>(gf, gc, T, xf, xc);
  else if (gf.k == 3) heat_restrict_kernel<3><<<grid_of(gc.ndofs), 256, 0, s>>>(gf, gc, T, xf, xc);
  else throw WrError(WR_ERR_ARG, "heat: k must be 1..3");
  WR_LAUNCH_CHECK();
}

void heat_prolong_add(const LevelGeom& gf, const LevelGeom& gc, const FeTables& T, const double* xc, double* xf,
                      cudaStream_t s) {
  if (gf.k == 1) heat_prolong_kernel<1><<<grid_of(gf.ndofs), 256, 0, s>>>(gf, gc, T, xc, xf);
  else if (gf.k == 2) heat_prolong_kernel<2><<<grid_of(gf.ndofs), 256, 0, s>>>(gf, gc, T, xc, xf);
  else if (gf.k == 3) heat_prolong_kernel<3><<<grid_of(gf.ndofs), 256, 0, s>>>(gf, gc, T, xc, xf);
  else throw WrError(WR_ERR_ARG, "heat: k must be 1..3");
  WR_LAUNCH_CHECK();
}

void heat_splitmix(int64_t n, uint64_t seed, double* x, cudaStream_t s) {
  heat_splitmix_kernel<<<grid_of(n), 256, 0, s>>>(n, seed, x);
  WR_LAUNCH_CHECK();
}

int heat_patch_slots(const LevelGeom& g, int blk, int* d_out, cudaStream_t s) {
  if (g.k == 1) heat_patch_slots_kernel<1><<<1, 32, 0, s>>>(g, blk, d_out);
  else if (g.k == 2) heat_patch_slots_kernel<2><<<1, 32, 0, s>>>(g, blk, d_out);
  else if (g.k == 3) heat_patch_slots_kernel<3><<<1, 32, 0, s>>>(g, blk, d_out);
  else throw WrError(WR_ERR_ARG, "heat: k must be 1..3");
  WR_LAUNCH_CHECK();
  return (2 * g.k - 1) * (2 * g.k - 1);
}
