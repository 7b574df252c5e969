// Waveform Vanka+star relaxation (hot-path steps (a)-(d)) and the coarse-level
// direct solve, which is the same block forward substitution on one block that
// holds every free DoF.
//
// Patches (Sec. 3, NS relaxation; Fig. patches): one per vertex (I, J).  Velocity
// slots form the (2k+3) x (2k+3) node grid of the closed 2x2-cell block around
// the vertex (the closure of the vertex star), per component; pressure slots the
// (2k-1) x (2k-1) grid of the open star.  Slots off the domain or on the
// Dirichlet boundary are padding: identity rows and columns, zero data.
//
// (b) block_factor_kernel, one CTA per (patch, slab): assembles the slab
//     diagonal block A_nn = J(W)[P_i, P_i] (principal submatrix of the
//     assembled space-time Jacobian) directly in shared memory from the global
//     1D mass/stiffness/divergence entries and the element convection matrices,
//     then inverts it.  For DG(1) the block has 2x2 temporal sub-blocks of size
//     ms <= 107; it is factored as
//         A00^{-1},  X = A00^{-1} A01,  S = A11 - A10 X,  S^{-1}
//     (block LU over the temporal DoFs, Gauss-Jordan with partial pivoting inside
//     each block), which keeps every working matrix inside shared memory.
// (a)+(c) block_apply_kernel, persistent CTAs, one patch at a time, sequential
//     over slabs: gathers r on the patch, adds the jump coupling
//     tau_a(0) M_u y_{n-1} (Eq. waveform_patch_solve: A_{n,n-1} = -tau_a(0) M_u on
//     the last temporal DoF's velocity), applies the stored factors, which are
//     streamed HBM -> shared memory by cp.async.bulk through an mbarrier ring.
// (d) scatter_kernel: every global DoF pulls the outputs of the patches that
//     contain it in a fixed order (deterministic weighted additive scatter, w = 1).
#include <cuda_bf16.h>

#include <cmath>

#include "wrmg_internal.h"

namespace {

// Slot shape of a block: velocity grid NVG x NVG per component, pressure grid
// NPG x NPG.  Patches: NVG = 2k+3, NPG = 2k-1; the coarse 2x2 block fits the
// patch shape; the coarse 3x3 block of Q2/Q1 uses NPG = 4 (5x5 velocity, 66 slots).
template <int K, int NPGX = 2 * K - 1>
struct PD {
  static constexpr int NVG = 2 * K + 3, NPG = NPGX;
  static constexpr int NVG2 = NVG * NVG;
  static constexpr int MS = 2 * NVG2 + NPG * NPG;         // 51 (k = 1) or 107 (k = 2)
  static constexpr int LD = (MS % 2) ? MS : MS + 1;       // odd leading dimension in smem
  static constexpr int NVL = K + 2, NVE = NVL * NVL;
};

// Sparsity of the off-diagonal temporal block A10 of a DG(1) patch block (kind 0), the
// one stored block that is not a factor but an assembled Jacobian block: two slots couple
// only if some cell contains both, and the slot grid spans exactly the patch's 2 x 2 cells
// (velocity slot x in the first cell along an axis if x <= K+1, in the second if x >= K+1;
// pressure slot x in the first if x <= K-1, in the second if x >= K-1), so two slots
// couple iff they share a cell along both axes and are not both pressure slots (the
// Taylor-Hood pressure block is zero): 41% of a Q3/Q2 block, 48% of a Q2/Q1 block.  Its
// rows are cut into segments of at most L entries; FP64 A10 blocks are stored by
// segments, item i of segment t at i * NSEGP + t (consecutive segments adjacent, so that
// a warp reads 32 consecutive values), items past a segment's end zero.
template <int K>
struct SpA10 {
  static constexpr int NVG = 2 * K + 3, NPG = 2 * K - 1, NV2 = NVG * NVG, MS = 2 * NV2 + NPG * NPG;
  static constexpr int L = K == 2 ? 36 : 19;  // entries per segment at most
  __host__ __device__ static constexpr bool vel(int s) { return s < 2 * NV2; }
  __host__ __device__ static constexpr int sx(int s) { return vel(s) ? s % NV2 % NVG : (s - 2 * NV2) % NPG; }
  __host__ __device__ static constexpr int sy(int s) { return vel(s) ? s % NV2 / NVG : (s - 2 * NV2) / NPG; }
  // bit 0: in the patch's first cell along an axis; bit 1: in its second
  __host__ __device__ static constexpr unsigned cells(bool v, int c) {
    return v ? ((c <= K + 1 ? 1u : 0u) | (c >= K + 1 ? 2u : 0u)) : ((c <= K - 1 ? 1u : 0u) | (c >= K - 1 ? 2u : 0u));
  }
  __host__ __device__ static constexpr bool couple(int a, int b) {
    return (vel(a) || vel(b)) && (cells(vel(a), sx(a)) & cells(vel(b), sx(b))) != 0u &&
           (cells(vel(a), sy(a)) & cells(vel(b), sy(b))) != 0u;
  }
  __host__ __device__ static constexpr int len(int r) {
    int n = 0;
    for (int c = 0; c < MS; ++c) n += couple(r, c) ? 1 : 0;
    return n;
  }
  __host__ __device__ static constexpr int count(bool segments) {
    int n = 0;
    for (int r = 0; r < MS; ++r) n += segments ? (len(r) + L - 1) / L : len(r);
    return n;
  }
  static constexpr int NSEG = count(true), NNZ = count(false);
  static constexpr int NSEGP = (NSEG + 31) / 32 * 32;  // segments padded to whole warps
  static constexpr int ELEMS = L * NSEGP;              // stored entries
};
static_assert(SpA10<2>::MS == 107 && SpA10<1>::MS == 51, "patch slot counts");
static_assert(SpA10<2>::NNZ == 4744 && SpA10<2>::NSEG == 141, "Q3/Q2 A10 pattern");
static_assert(SpA10<1>::NNZ == 1256 && SpA10<1>::NSEG == 73, "Q2/Q1 A10 pattern");

// The segment tables: row and length of each segment, column of each item (0 past the
// segment's end), first segment and segment count of each row.
template <int K>
struct SpTab {
  short col[SpA10<K>::ELEMS];
  short seg_row[SpA10<K>::NSEGP], seg_len[SpA10<K>::NSEGP];
  short start[SpA10<K>::MS], nseg[SpA10<K>::MS];
};
template <int K>
constexpr SpTab<K> make_sp_tab() {
  using S = SpA10<K>;
  SpTab<K> t{};
  int acc = 0;
  for (int r = 0; r < S::MS; ++r) {
    const int n = S::len(r), ns = (n + S::L - 1) / S::L;
    t.start[r] = (short)acc;
    t.nseg[r] = (short)ns;
    for (int j = 0; j < ns; ++j) {
      t.seg_row[acc + j] = (short)r;
      t.seg_len[acc + j] = (short)(n - j * S::L < S::L ? n - j * S::L : S::L);
    }
    int k = 0;
    for (int c = 0; c < S::MS; ++c)
      if (S::couple(r, c)) {
        t.col[(k % S::L) * S::NSEGP + acc + k / S::L] = (short)c;
        ++k;
      }
    acc += ns;
  }
  return t;
}
__device__ const SpTab<1> g_sp1 = make_sp_tab<1>();
__device__ const SpTab<2> g_sp2 = make_sp_tab<2>();
template <int K>
__device__ __forceinline__ const SpTab<K>& sp_tab() {
  if constexpr (K == 1) return g_sp1;
  else return g_sp2;
}

// Layout of one stored factor block (MS x MS): column-major with leading dimension MS,
// padded to a 16-byte granule, except the FP32 and BF16 blocks of Q2/Q1 patches
// (MS = 51): their first CG = 48 columns are stored by groups of GV = 16 bytes / entry
// (4 FP32 or 8 BF16 entries) -- entry (i, j) at ((j / GV) MS + i) GV + j % GV, so that the
// entries of row i in one group of columns share one 16-byte word (one load for GV FMAs
// in the warp tiles) -- and their last MS - CG columns follow column-major.
template <typename FT, int MS>
struct Stored {
  static constexpr int GV = (sizeof(FT) <= 4 && MS < 64) ? 16 / (int)sizeof(FT) : 1;
  static constexpr bool GRP = GV > 1;
  static constexpr int GR = 16 / (int)sizeof(FT);
  static constexpr int CG = GRP ? MS / GV * GV : 0;  // columns stored by groups
  static constexpr int BLK = (MS * MS + GR - 1) / GR * GR;
  __host__ __device__ static constexpr int at(int i, int j) {
    if constexpr (!GRP) return j * MS + i;
    else return j < CG ? ((j / GV) * MS + i) * GV + j % GV : CG * MS + (j - CG) * MS + i;
  }
};
// the two BF16 entries of a 32-bit word, widened exactly to FP32
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
// acc + sum_j A_j x_j over one 16-byte group of a row, in column order (one FMA chain):
// 8 BF16 entries against xa, xb, or 4 FP32 entries against xa
template <typename FT>
__device__ __forceinline__ float grp_fma(const uint4 w, const float4 xa, const float4 xb, float acc) {
  if constexpr (sizeof(FT) == 2) {
    acc = fmaf(bf16_lo(w.x), xa.x, acc);
    acc = fmaf(bf16_hi(w.x), xa.y, acc);
    acc = fmaf(bf16_lo(w.y), xa.z, acc);
    acc = fmaf(bf16_hi(w.y), xa.w, acc);
    acc = fmaf(bf16_lo(w.z), xb.x, acc);
    acc = fmaf(bf16_hi(w.z), xb.y, acc);
    acc = fmaf(bf16_lo(w.w), xb.z, acc);
    return fmaf(bf16_hi(w.w), xb.w, acc);
  } else {
    (void)xb;
    acc = fmaf(__uint_as_float(w.x), xa.x, acc);
    acc = fmaf(__uint_as_float(w.y), xa.y, acc);
    acc = fmaf(__uint_as_float(w.z), xa.z, acc);
    return fmaf(__uint_as_float(w.w), xa.w, acc);
  }
}
// the input entries of one group of columns (x 16-byte aligned)
template <typename FT>
__device__ __forceinline__ void grp_x(const float* x, float4& xa, float4& xb) {
  xa = *reinterpret_cast<const float4*>(x);
  if constexpr (sizeof(FT) == 2) xb = *reinterpret_cast<const float4*>(x + 4);
  else xb = xa;
}

// Block LDU of a slab's diagonal block over its NT = q+1 temporal sub-blocks (block
// Gaussian elimination without pivoting across sub-blocks, partial pivoting inside the
// diagonal ones):  S_k = A_kk - sum_{m<k} C_km X_mk,  C_ik = A_ik - sum_{m<k} C_im X_mk
// (i > k),  X_kj = S_k^{-1} (A_kj - sum_{m<k} C_km X_mj) (j > k).  The NT^2 stored
// blocks S_k^{-1}, C_ik, X_kj are kept in the order the apply consumes them:
//   forward, k = 0 .. NT-1:   z_k = S_k^{-1} r_k;  r_i -= C_ik z_k (i = k+1 .. NT-1)
//   backward, k = NT-2 .. 0:  y_k -= X_kj y_j (j = k+1 .. NT-1), with y_k = z_k before.
// DG(0) is the single inverse; DG(1) is [A00^{-1}, A10, S^{-1}, X].
struct BlockOp {
  int src_y, src;  // source vector: y (1) or the right-hand side r (0), temporal index
  int dst, di;     // 0: y_di = result, 1: r_di -= result, 2: y_di -= result
};
template <int NT>
__host__ __device__ constexpr BlockOp block_op(int b) {
  constexpr int nf = NT * (NT + 1) / 2;  // forward blocks
  BlockOp o{0, 0, 0, 0};
  if (b < nf) {
    int k = 0, base = 0;
    while (b >= base + (NT - k)) {
      base += NT - k;
      ++k;
    }
    const int r = b - base;
    if (r == 0) o = BlockOp{0, k, 0, k};
    else o = BlockOp{1, k, 1, k + r};
  } else {
    int rem = b - nf, k = NT - 2;
    while (rem >= NT - 1 - k) {
      rem -= NT - 1 - k;
      --k;
    }
    o = BlockOp{1, k + 1 + rem, 2, k};
  }
  return o;
}
// storage positions of S_k^{-1}, C_ik (i > k) and X_kj (j > k)
template <int NT>
__host__ __device__ constexpr int pos_diag(int k) { return k * NT - k * (k - 1) / 2; }
template <int NT>
__host__ __device__ constexpr int pos_low(int i, int k) { return pos_diag<NT>(k) + (i - k); }
template <int NT>
__host__ __device__ constexpr int pos_up(int k, int j) {
  return NT * (NT + 1) / 2 + (NT - 2 - k) * (NT - 1 - k) / 2 + (j - k - 1);
}
static_assert(pos_diag<2>(1) == 2 && pos_low<2>(1, 0) == 1 && pos_up<2>(0, 1) == 3, "DG(1) block order");
static_assert(block_op<3>(6).dst == 2 && block_op<3>(6).di == 1 && block_op<3>(6).src == 2, "DG(2) block order");
static_assert(pos_up<4>(0, 3) == 15 && pos_up<4>(2, 3) == 10 && pos_low<4>(3, 2) == 8, "DG(3) block order");

struct Slot {
  int field;   // 0, 1 velocity component, 2 pressure
  int gx, gy;  // global node
  int sp;      // spatial index within a temporal block, -1 = padding
};

__device__ __forceinline__ void block_origin(const LevelGeom& g, const BlockSet& bs, int blk, int& vx0, int& vy0,
                                             int& px0, int& py0) {
  if (bs.kind == 0) {
    const int I = blk % (g.n + 1), J = blk / (g.n + 1);
    vx0 = (I - 1) * (g.k + 1);
    vy0 = (J - 1) * (g.k + 1);
    px0 = I * g.k - (g.k - 1);
    py0 = J * g.k - (g.k - 1);
  } else {
    vx0 = vy0 = 1;
    px0 = py0 = 0;
  }
}

// 1D cell range [c0, c0 + 1] of the 2x2 cell block of a patch (kind 0) along one
// direction, from the block's first velocity node v0 = (I - 1)(k + 1); the whole
// mesh when the patch system is the principal submatrix or the block is not a patch.
__device__ __forceinline__ void own_cells(const LevelGeom& g, const BlockSet& bs, int v0, int& c0, int& c1) {
  if (bs.kind == 0 && bs.local) {
    c0 = v0 / (g.k + 1);  // exact: v0 is a multiple of k + 1 (c0 = -1 for I = 0)
    c1 = c0 + 1;
  } else {
    c0 = 0;
    c1 = 1 << 30;
  }
}

__device__ __forceinline__ Slot decode_slot(const LevelGeom& g, const BlockSet& bs, int blk, int s) {
  int vx0, vy0, px0, py0;
  block_origin(g, bs, blk, vx0, vy0, px0, py0);
  const int nv2g = bs.nvg * bs.nvg;
  Slot r;
  r.sp = -1;
  if (s < 2 * nv2g) {
    r.field = s / nv2g;
    const int t = s % nv2g;
    r.gx = vx0 + t % bs.nvg;
    r.gy = vy0 + t / bs.nvg;
    if (r.gx >= 1 && r.gx <= g.nv - 2 && r.gy >= 1 && r.gy <= g.nv - 2)
      r.sp = r.field * g.nv * g.nv + r.gy * g.nv + r.gx;
  } else if (s < 2 * nv2g + bs.npg * bs.npg) {
    r.field = 2;
    const int t = s - 2 * nv2g;
    r.gx = px0 + t % bs.npg;
    r.gy = py0 + t / bs.npg;
    const bool pinned = bs.kind == 1 && r.gx == 0 && r.gy == 0;
    if (r.gx >= 0 && r.gx < g.np && r.gy >= 0 && r.gy < g.np && !pinned)
      r.sp = 2 * g.nv * g.nv + r.gy * g.np + r.gx;
  } else {
    r.field = 3;
    r.gx = r.gy = 0;
  }
  return r;
}

// cells [lo, hi] of the 1D mesh containing node g of a degree-p Lagrange space
__device__ __forceinline__ int cell_lo(int g, int p) { return g == 0 ? 0 : (g - 1) / p; }
__device__ __forceinline__ int cell_hi(int g, int p, int n) { return min(g / p, n - 1); }

// global 1D velocity-velocity matrix entry sum_c ref[gi - pc][gj - pc], over the
// cells c in [clo, chi] only (the whole mesh by default)
template <int K>
__device__ __forceinline__ double vv1(const double (*ref)[WR_MAX_NVL], int n, int gi, int gj, int clo = 0,
                                      int chi = 1 << 30) {
  const int p = K + 1;
  const int lo = max(max(cell_lo(gi, p), cell_lo(gj, p)), clo);
  const int hi = min(min(cell_hi(gi, p, n), cell_hi(gj, p, n)), chi);
  double v = 0.0;
  for (int c = lo; c <= hi; ++c) v += ref[gi - p * c][gj - p * c];
  return v;
}
// global 1D pressure-velocity entry sum_c ref[pn - kc][vn - (k+1)c]
template <int K>
__device__ __forceinline__ double pv1(const double (*ref)[WR_MAX_NVL], int n, int pn, int vn) {
  const int lo = max(cell_lo(pn, K), cell_lo(vn, K + 1)), hi = min(cell_hi(pn, K, n), cell_hi(vn, K + 1, n));
  double v = 0.0;
  for (int c = lo; c <= hi; ++c) v += ref[pn - K * c][vn - (K + 1) * c];
  return v;
}

// ---------------------------------------------------------------- factorisation
// One CTA per (block, slab).  The slab diagonal block A_nn = J(W)[P_i, P_i] is
// assembled in shared memory in two passes per temporal sub-block (a, b):
//   1. the constant-coefficient part from per-patch tables of the global 1D
//      matrices restricted to the slot grid (tensor products on the Cartesian
//      mesh):  Kt[a,b] M + dt nu Wt[a,b] K  on velocity pairs of one component,
//      dt Wt[a,b] (chi, d_c phi) on velocity-pressure pairs;
//   2. the convection  dt conv sum_e T3[a,b,e] Ce_e  scattered cell by cell from
//      the element convection matrices of every cell whose closure meets the
//      slot grid (the 2x2 star and, for the principal submatrix, its ring of
//      cells), with coalesced reads and no write conflicts.
// The block is then inverted by Gauss-Jordan with partial pivoting (DG(0)), or,
// for DG(1), factored as A00^{-1}, X = A00^{-1} A01, S = A11 - A10 X, S^{-1}.
// CT is the arithmetic and storage type: double (plain form) or float
// (precision form; FP32 runs at 58x the FP64 rate on GB300).

// The threads that build one block: the whole CTA, or one warp of it.
struct CtaGroup {
  int t, n;  // this thread's index in the group, group size
  __device__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
  int t, n;
  __device__ void sync() const { __syncwarp(); }
};

// Per-block tables of the global 1D matrices on the slot grid, in the assembly's
// arithmetic type VT (computed in FP64, rounded once to VT).
template <int K, int NPGX = 2 * K - 1, typename VT = double>
struct FactorTables {
  static constexpr int NVG = 2 * K + 3;
  static constexpr int NPT = 2 * K + 1 > NPGX ? 2 * K + 1 : NPGX;  // pressure rows (coarse blocks are larger)
  VT Mx[NVG][NVG], Kx[NVG][NVG], My[NVG][NVG], Ky[NVG][NVG];
  VT Dx[NPT][NVG], Cx[NPT][NVG], Dy[NPT][NVG], Cy[NPT][NVG];
  signed char sf[PD<K, NPGX>::MS];                   // slot field 0/1 velocity, 2 pressure, -1 padding
  signed char sx[PD<K, NPGX>::MS], sy[PD<K, NPGX>::MS];  // slot-grid coordinates
};

template <int K, int NPGX, typename VT, class Grp>
__device__ void build_factor_tables(const LevelGeom& g, const FeTables& T, const BlockSet& bs, int blk,
                                    FactorTables<K, NPGX, VT>& ft, const Grp& gr) {
  using pd = PD<K, NPGX>;
  using TB = FactorTables<K, NPGX, VT>;
  int vx0, vy0, px0, py0;
  block_origin(g, bs, blk, vx0, vy0, px0, py0);
  const double h = g.h;
  int cx0, cx1, cy0, cy1;
  own_cells(g, bs, vx0, cx0, cx1);
  own_cells(g, bs, vy0, cy0, cy1);
  for (int e = gr.t; e < TB::NVG * TB::NVG; e += gr.n) {
    const int i = e / TB::NVG, j = e % TB::NVG;
    const int xi = min(max(vx0 + i, 0), g.nv - 1), xj = min(max(vx0 + j, 0), g.nv - 1);
    const int yi = min(max(vy0 + i, 0), g.nv - 1), yj = min(max(vy0 + j, 0), g.nv - 1);
    ft.Mx[i][j] = (VT)(h * vv1<K>(T.m1, g.n, xi, xj, cx0, cx1));
    ft.Kx[i][j] = (VT)(vv1<K>(T.k1, g.n, xi, xj, cx0, cx1) / h);
    ft.My[i][j] = (VT)(h * vv1<K>(T.m1, g.n, yi, yj, cy0, cy1));
    ft.Ky[i][j] = (VT)(vv1<K>(T.k1, g.n, yi, yj, cy0, cy1) / h);
  }
  for (int e = gr.t; e < TB::NPT * TB::NVG; e += gr.n) {
    const int p = e / TB::NVG, v = e % TB::NVG;
    const int pxg = min(max(px0 + p, 0), g.np - 1), pyg = min(max(py0 + p, 0), g.np - 1);
    const int vxg = min(max(vx0 + v, 0), g.nv - 1), vyg = min(max(vy0 + v, 0), g.nv - 1);
    ft.Dx[p][v] = (VT)pv1<K>(T.d1, g.n, pxg, vxg);
    ft.Cx[p][v] = (VT)(h * pv1<K>(T.c1, g.n, pxg, vxg));
    ft.Dy[p][v] = (VT)pv1<K>(T.d1, g.n, pyg, vyg);
    ft.Cy[p][v] = (VT)(h * pv1<K>(T.c1, g.n, pyg, vyg));
  }
  for (int s = gr.t; s < pd::MS; s += gr.n) {
    const Slot sl = decode_slot(g, bs, blk, s);
    if (sl.sp < 0) {
      ft.sf[s] = -1;
      ft.sx[s] = ft.sy[s] = 0;
    } else if (sl.field < 2) {
      ft.sf[s] = (signed char)sl.field;
      ft.sx[s] = (signed char)(sl.gx - vx0);
      ft.sy[s] = (signed char)(sl.gy - vy0);
    } else {
      ft.sf[s] = 2;
      ft.sx[s] = (signed char)(sl.gx - px0);
      ft.sy[s] = (signed char)(sl.gy - py0);
    }
  }
}

// M (+)= constant part of temporal sub-block (a, b); padding rows/columns get the identity on a == b.
// Arithmetic in CT (FP64 for the plain form, FP32 for the reduced-precision ones).
template <int K, int Q, typename CT, int LD, int NPGX, class Grp>
__device__ void assemble_const(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                               const FactorTables<K, NPGX, CT>& ft, CT* M, int a, int b, bool add, const Grp& gr) {
  constexpr int MS = PD<K, NPGX>::MS;
  const CT kt = (CT)T.Kt[a][b], vis = (CT)(g.dt * ph.nu * T.Wt[a][b]), dw = (CT)(g.dt * T.Wt[a][b]);
  for (int e = gr.t; e < MS * MS; e += gr.n) {
    const int i = e / MS, j = e - (e / MS) * MS;
    const int fi = ft.sf[i], fj = ft.sf[j];
    CT v = 0;
    if (fi < 0 || fj < 0) {
      v = (i == j && a == b) ? CT(1) : CT(0);
    } else if (fi < 2 && fj < 2) {
      if (fi == fj) {
        const int ix = ft.sx[i], iy = ft.sy[i], jx = ft.sx[j], jy = ft.sy[j];
        const CT mx = ft.Mx[ix][jx], my = ft.My[iy][jy];
        v = kt * mx * my + vis * (ft.Kx[ix][jx] * my + mx * ft.Ky[iy][jy]);
      }
    } else if (fi < 2 || fj < 2) {
      const int sv = fi < 2 ? i : j, sq = fi < 2 ? j : i;
      const int c = ft.sf[sv];
      const int vx = ft.sx[sv], vy = ft.sy[sv], qx = ft.sx[sq], qy = ft.sy[sq];
      v = dw * (c == 0 ? ft.Dx[qx][vx] * ft.Cy[qy][vy] : ft.Cx[qx][vx] * ft.Dy[qy][vy]);
    }
    if (add)
      M[i * LD + j] += v;
    else
      M[i * LD + j] = v;
  }
}

// M += dt conv sum_e T3[a,b,e] Ce_e, cell by cell (one cell per pass: no write conflicts).
template <int K, int Q, typename CT, int LD, int NPGX, class Grp>
__device__ void assemble_conv(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const BlockSet& bs,
                              const CT* __restrict__ Ce, int blk, int slab, const FactorTables<K, NPGX, CT>& ft,
                              CT* M, int a, int b, const Grp& gr) {
  using pd = PD<K, NPGX>;
  constexpr int NT = Q + 1, NVL = pd::NVL, NVE = pd::NVE, NVG = pd::NVG;
  constexpr int MS = pd::MS;
  int vx0, vy0, px0, py0;
  block_origin(g, bs, blk, vx0, vy0, px0, py0);
  const int nvg = bs.nvg;
  // cells whose closure meets the slot grid (only the patch's own 2x2 cells when
  // the patch system is assembled over them)
  int cx0 = max(0, (vx0 - 1) / (K + 1) - (vx0 - 1 < 0 ? 1 : 0)), cx1 = min(g.n - 1, (vx0 + nvg - 1) / (K + 1));
  int cy0 = max(0, (vy0 - 1) / (K + 1) - (vy0 - 1 < 0 ? 1 : 0)), cy1 = min(g.n - 1, (vy0 + nvg - 1) / (K + 1));
  if (bs.kind == 0 && bs.local) {
    int a0, a1;
    own_cells(g, bs, vx0, a0, a1);
    cx0 = max(cx0, a0);
    cx1 = min(cx1, a1);
    own_cells(g, bs, vy0, a0, a1);
    cy0 = max(cy0, a0);
    cy1 = min(cy1, a1);
  }
  const double sc = g.dt * ph.conv;
  CT w[NT];
#pragma unroll
  for (int e = 0; e < NT; ++e) w[e] = (CT)(sc * T.T3[a][b][e]);
  for (int cy = cy0; cy <= cy1; ++cy)
    for (int cx = cx0; cx <= cx1; ++cx) {
      const CT* ce = Ce + ((int64_t)slab * g.ncells() + cy * g.n + cx) * (NT * 4 * NVE * NVE);
      for (int e = gr.t; e < 4 * NVE * NVE; e += gr.n) {
        const int cd = e / (NVE * NVE), r = e % (NVE * NVE);
        const int li = r / NVE, lj = r % NVE;
        const int ix = cx * (K + 1) + li % NVL - vx0, iy = cy * (K + 1) + li / NVL - vy0;
        const int jx = cx * (K + 1) + lj % NVL - vx0, jy = cy * (K + 1) + lj / NVL - vy0;
        if (ix < 0 || ix >= nvg || iy < 0 || iy >= nvg || jx < 0 || jx >= nvg || jy < 0 || jy >= nvg) continue;
        const int si = (cd >> 1) * nvg * nvg + iy * nvg + ix, sj = (cd & 1) * nvg * nvg + jy * nvg + jx;
        if (ft.sf[si] < 0 || ft.sf[sj] < 0) continue;
        CT v = 0;
#pragma unroll
        for (int ee = 0; ee < NT; ++ee) v += w[ee] * ce[(int64_t)ee * 4 * NVE * NVE + e];
        M[si * LD + sj] += v;
      }
      gr.sync();
    }
  (void)MS;
  (void)NVG;
}

// In-place Gauss-Jordan inversion with partial pivoting (largest |.|, lowest
// row on ties) of the MS x MS row-major matrix A (leading dimension LD) in
// shared memory.  Returns false (to all threads) if a zero (or non-finite) pivot
// was met.  Written to keep the FP64 pipe for the elimination itself (on GB300 it
// runs 2 FMA/clk/SM): the pivot search compares |x| as integer keys (the sign-
// cleared bit pattern orders finite values like |x|) on the integer pipe; the
// pivot's reciprocal is formed once, by the thread that picks the pivot; and every
// element of a step is one FMA: column p is pre-set to -0 (and the pivot entry of
// the scaled pivot row to the reciprocal), so that fma(-c_i, inv, -0) forms the
// new column exactly as the product -c_i inv would, without a divergent branch.
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned abs_key(float v) { return (unsigned)__float_as_int(v) & 0x7fffffffu; }

template <int MS, int LD, int NTH, typename CT>
__device__ bool gauss_jordan(CT* A, CT* colbuf, int* perm, int* sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  using Key = decltype(abs_key(CT(0)));
  __shared__ CT pinv;
#pragma unroll 1
  for (int p = 0; p < MS; ++p) {
    if (warp == 0) {
      Key best = 0;
      int bi = MS;
      for (int i = p + lane; i < MS; i += 32) {
        const Key v = abs_key(A[i * LD + p]);
        if (v > best || bi == MS) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const Key ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        sh[0] = bi;
        perm[p] = bi;
        const CT pv = A[bi * LD + p];  // the pivot, before the row exchange
        if (!(fabs(pv) > CT(0)) || !isfinite(pv)) sh[1] = 1;
        pinv = CT(1) / pv;
      }
    }
    __syncthreads();
    const int r = sh[0];
    if (r != p)
      for (int j = tid; j < MS; j += NTH) {
        const CT t = A[p * LD + j];
        A[p * LD + j] = A[r * LD + j];
        A[r * LD + j] = t;
      }
    __syncthreads();
    const CT inv = pinv;
    for (int i = tid; i < MS; i += NTH) {
      colbuf[i] = A[i * LD + p];
      if (i != p) A[i * LD + p] = CT(-0.0);
    }
    __syncthreads();
    for (int j = tid; j < MS; j += NTH) A[p * LD + j] = (j == p) ? inv : A[p * LD + j] * inv;
    __syncthreads();
    for (int e = tid; e < MS * MS; e += NTH) {
      const int i = e / MS, j = e - (e / MS) * MS;
      if (i == p) continue;
      A[i * LD + j] = fma(-colbuf[i], A[p * LD + j], A[i * LD + j]);
    }
    __syncthreads();
  }
#pragma unroll 1
  for (int p = MS - 1; p >= 0; --p) {
    const int r = perm[p];
    if (r != p)
      for (int i = tid; i < MS; i += NTH) {
        const CT t = A[i * LD + p];
        A[i * LD + p] = A[i * LD + r];
        A[i * LD + r] = t;
      }
    __syncthreads();
  }
  return sh[1] == 0;
}

// Register-tiled Gauss-Jordan inversion with partial pivoting, the same elimination
// as gauss_jordan above without moving rows: thread (ty, tx) of a (NTH/32) x 32 grid
// holds rows ty + TY u and columns tx + 32 v of A in registers for the whole
// inversion.  Per pivot column p: the column goes to shared memory, every warp picks
// the pivot row (largest |.| among rows not yet used, compared to 16 mantissa bits,
// lowest row on ties), the warp that owns that row publishes it scaled, and every
// thread updates its own entries (two block barriers per pivot; the column and row
// buffers alternate between pivots, and the used-row flags change only after the
// second barrier).  The inverse is read back with the pivot order undone:
// inv(A)[i][r_q] = X[r_i][q] for the pivot rows r.  A is MS x MS row-major with
// leading dimension LD in shared memory, overwritten with inv(A).  Returns false (to
// all threads) if a zero pivot was met.
template <int MS, int LD, int NTH, typename CT>
__device__ bool gauss_jordan_reg(CT* A) {
  constexpr int TY = NTH / 32, RU = (MS + TY - 1) / TY, CV = (MS + 31) / 32;
  static_assert(sizeof(CT) == 4 && MS <= 128, "pivot keys hold an FP32 |x| and a row below 128");
  __shared__ CT colb[2][MS], rowb[2][MS];
  __shared__ int used[MS], prow[MS], pstep[MS], zero_pivot;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  CT a[RU][CV];
#pragma unroll
  for (int u = 0; u < RU; ++u)
#pragma unroll
    for (int v = 0; v < CV; ++v) {
      const int i = ty + TY * u, j = lane + 32 * v;
      a[u][v] = (i < MS && j < MS) ? A[i * LD + j] : CT(0);
    }
  for (int i = tid; i < MS; i += NTH) used[i] = 0;
  if (tid == 0) zero_pivot = 0;
  __syncthreads();
  // pivots in groups of 32 so that the register column of pivot p (p / 32) is a constant
#pragma unroll
  for (int vp = 0; vp < CV; ++vp) {
#pragma unroll 1
    for (int p = 32 * vp; p < MS && p < 32 * vp + 32; ++p) {
      const int bsel = p & 1;
      // column p to shared memory (owned by the lanes with lane == p % 32), then set to
      // -0 there: fma(-f, inv, -0) below forms the new column p, -f inv, exactly
      if (lane == (p & 31)) {
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const int i = ty + TY * u;
          if (i < MS) colb[bsel][i] = a[u][vp];
          a[u][vp] = CT(-0.0);
        }
      }
      __syncthreads();
      // every warp finds the same pivot row: one integer max over keys that hold |x|
      // to 16 mantissa bits above 127 - row (rows already used have key 0)
      unsigned key = 0u;
      for (int i = lane; i < MS; i += 32)
        if (!used[i]) key = max(key, (abs_key(colb[bsel][i]) & 0x7fffff80u) | (unsigned)(127 - i));
      key = __reduce_max_sync(0xffffffffu, key);
      const int r = 127 - (int)(key & 127u);
      const CT pv = colb[bsel][r];
      const CT inv = CT(1) / pv;
      // the owner warp of row r publishes it scaled by the inverse pivot
      if (ty == r % TY) {
        const int ur = r / TY;
#pragma unroll
        for (int v = 0; v < CV; ++v) {
          CT val = CT(0);
#pragma unroll
          for (int u = 0; u < RU; ++u) val = (u == ur) ? a[u][v] : val;
          const int j = lane + 32 * v;
          if (j < MS) rowb[bsel][j] = (j == p) ? inv : val * inv;
        }
      }
      __syncthreads();
      // rank-one update of every row but the pivot row (its multiplier is zero), which
      // its owner warp then overwrites with the published row
      CT rj[CV];
#pragma unroll
      for (int v = 0; v < CV; ++v) {
        const int j = lane + 32 * v;
        rj[v] = j < MS ? rowb[bsel][j] : CT(0);
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int i = ty + TY * u;
        const CT f = (i < MS && i != r) ? colb[bsel][i] : CT(0);
#pragma unroll
        for (int v = 0; v < CV; ++v) a[u][v] = fma(-f, rj[v], a[u][v]);
      }
      if (ty == r % TY) {
        const int ur = r / TY;
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int v = 0; v < CV; ++v) a[u][v] = (u == ur) ? rj[v] : a[u][v];
      }
      // bookkeeping after the second barrier, so that no warp's search of this pivot sees it
      if (tid == 0) {
        used[r] = 1;
        prow[p] = r;
        pstep[r] = p;
        if (!(fabs(pv) > CT(0))) zero_pivot = 1;
      }
    }
  }
  __syncthreads();
  // undo the pivot order: inv(A)[pstep[row]][prow[col]] = X[row][col]
#pragma unroll
  for (int u = 0; u < RU; ++u)
#pragma unroll
    for (int v = 0; v < CV; ++v) {
      const int i = ty + TY * u, j = lane + 32 * v;
      if (i < MS && j < MS) A[pstep[i] * LD + prow[j]] = a[u][v];
    }
  __syncthreads();
  return zero_pivot == 0;
}


// Block inversion for the factor kernel.  FP64 keeps the shared-memory form: the FP64
// pipe bounds it, and the register tile's padding to (NTH/32) x 32 multiples costs
// 25-38% more FMAs (measured 6.5 s vs 9.0 s for the 64 x 64 Q3/Q2 DG(1) hierarchy);
// FP32 takes the register tile, which removes the shared-memory round trips that
// bound it (2.9 s vs 2.2 s).
template <int MS, int LD, int NTH, typename CT>
__device__ bool invert_block(CT* A, CT* colbuf, int* perm, int* sh) {
  if constexpr (sizeof(CT) == 8) {
    return gauss_jordan<MS, LD, NTH>(A, colbuf, perm, sh);
  } else {
    (void)colbuf; (void)perm; (void)sh;
    return gauss_jordan_reg<MS, LD, NTH>(A);
  }
}

__device__ __forceinline__ void narrow(double v, double& d) { d = v; }
__device__ __forceinline__ void narrow(float v, float& d) { d = v; }
__device__ __forceinline__ void narrow(float v, __nv_bfloat16& d) { d = __float2bfloat16_rn(v); }

template <int MS, int LD, int NTH, typename CT, typename ST>
__device__ void store_colmajor(const CT* A, ST* dst) {
  using SL = Stored<ST, MS>;
  if constexpr (SL::GRP) {
    for (int e = threadIdx.x; e < MS * MS; e += NTH) {
      int i, j;
      if (e < SL::CG * MS) {
        const int o = e / (MS * SL::GV), rem = e - o * (MS * SL::GV);
        i = rem / SL::GV;
        j = o * SL::GV + rem % SL::GV;
      } else {
        const int t = e - SL::CG * MS;
        j = SL::CG + t / MS;
        i = t - (j - SL::CG) * MS;
      }
      narrow(A[i * LD + j], dst[e]);
    }
  } else {
    for (int e = threadIdx.x; e < MS * MS; e += NTH) {
      const int j = e / MS, i = e - j * MS;
      narrow(A[i * LD + j], dst[e]);
    }
  }
}

// A (MS x MS, row-major, leading dimension LD) stored by the segments of SpA10<K>.
template <int K, int MS, int LD, int NTH, typename CT, typename ST>
__device__ void store_sparse_a10(const CT* A, ST* dst) {
  using S = SpA10<K>;
  static_assert(S::MS == MS, "A10 slot count");
  const SpTab<K>& tb = sp_tab<K>();
  for (int e = threadIdx.x; e < S::ELEMS; e += NTH) {
    const int i = e / S::NSEGP, t = e - i * S::NSEGP;
    narrow(i < tb.seg_len[t] ? A[tb.seg_row[t] * LD + tb.col[e]] : CT(0), dst[e]);
  }
}

// M -= P Q for an MS x MS shared-memory M (row-major, leading dimension LD) and P, Q
// stored blocks in global memory (column-major, leading dimension MS) that this CTA
// wrote before its last barrier.
template <int MS, int LD, int NTH, typename CT, typename ST>
__device__ void gemm_sub_stored(CT* M, const ST* P, const ST* Qm) {
  static_assert(!Stored<ST, MS>::GRP, "stored blocks read back column-major");
  for (int e = threadIdx.x; e < MS * MS; e += NTH) {
    const int i = e / MS, j = e - i * MS;
    CT acc = 0;
#pragma unroll 4
    for (int l = 0; l < MS; ++l) acc = fma((CT)P[l * MS + i], (CT)Qm[j * MS + l], acc);
    M[i * LD + j] -= acc;
  }
  __syncthreads();
}

// C = sign * A B (+ C if accumulate) for MS x MS shared-memory matrices, result written over B.
template <int MS, int LD, int NTH, typename CT>
__device__ void gemm_into_b(const CT* A, CT* B, CT sign) {
  constexpr int NE = (MS * MS + NTH - 1) / NTH;
  CT acc[NE];
  int ioff[NE], jcol[NE];
#pragma unroll
  for (int t = 0; t < NE; ++t) {
    const int e = threadIdx.x + t * NTH;
    const int i = e < MS * MS ? e / MS : 0;
    ioff[t] = i * LD;
    jcol[t] = e < MS * MS ? e - i * MS : 0;
    acc[t] = 0;
  }
#pragma unroll 1
  for (int l = 0; l < MS; ++l)
#pragma unroll
    for (int t = 0; t < NE; ++t) acc[t] = fma(A[ioff[t] + l], B[l * LD + jcol[t]], acc[t]);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NE; ++t)
    if (threadIdx.x + t * NTH < MS * MS) B[ioff[t] + jcol[t]] = sign * acc[t];
  __syncthreads();
}

// The same product for the reduced-precision forms, register-tiled like gauss_jordan_reg:
// thread (ty, tx) of the (NTH/32) x 32 grid accumulates rows ty + TY u and columns
// tx + 32 v, so per k it loads RU entries of A (one address per warp) and CV of B (32
// consecutive entries per warp) for RU x CV FMAs, at offsets fixed at compile time.  Each
// output entry is the same FMA chain over k = 0 .. MS-1 as in gemm_into_b (bitwise the
// same result); rows and columns past MS read row / column MS-1 and are not stored.
template <int MS, int LD, int NTH, typename CT>
__device__ void gemm_into_b_reg(const CT* A, CT* B, CT sign) {
  constexpr int TY = NTH / 32, RU = (MS + TY - 1) / TY, CV = (MS + 31) / 32;
  const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
  CT acc[RU][CV];
  const CT* arow[RU];
  int bcol[CV];
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    const int i = ty + TY * u;
    arow[u] = A + (i < MS ? i : MS - 1) * LD;
#pragma unroll
    for (int v = 0; v < CV; ++v) acc[u][v] = CT(0);
  }
#pragma unroll
  for (int v = 0; v < CV; ++v) {
    const int j = lane + 32 * v;
    bcol[v] = j < MS ? j : MS - 1;
  }
#pragma unroll 2
  for (int l = 0; l < MS; ++l) {
    CT av[RU], bv[CV];
#pragma unroll
    for (int u = 0; u < RU; ++u) av[u] = arow[u][l];
#pragma unroll
    for (int v = 0; v < CV; ++v) bv[v] = B[l * LD + bcol[v]];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < CV; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < RU; ++u)
#pragma unroll
    for (int v = 0; v < CV; ++v) {
      const int i = ty + TY * u, j = lane + 32 * v;
      if (i < MS && j < MS) B[i * LD + j] = sign * acc[u][v];
    }
  __syncthreads();
}

// B = sign A B for the factor kernel: FP64 keeps gemm_into_b (its 128-register budget
// holds the per-entry indices, and the FP64 pipe bounds it); FP32 takes the register tile,
// which under the 64-register budget of two CTAs per SM needs no index recomputation.
template <int MS, int LD, int NTH, typename CT>
__device__ void gemm_block(const CT* A, CT* B, CT sign) {
  if constexpr (sizeof(CT) == 8) gemm_into_b<MS, LD, NTH, CT>(A, B, sign);
  else gemm_into_b_reg<MS, LD, NTH, CT>(A, B, sign);
}

// Two CTAs per SM for the reduced-precision Q3/Q2 blocks (64 registers; the register-
// tiled inversion is latency-bound, so a second CTA hides its barriers); FP64 Q3/Q2
// needs 183 KB of shared memory and runs one.
template <int K, int Q, typename CT, typename ST, int NTH, int NPGX>
__global__ void __launch_bounds__(NTH, (sizeof(CT) == 4 && K == 2) ? 2 : 1)
block_factor_kernel(LevelGeom g, FeTables T, PhysParams ph, BlockSet bs, const CT* __restrict__ Ce,
                    ST* __restrict__ factors, int* __restrict__ status) {
  using pd = PD<K, NPGX>;
  constexpr int MS = pd::MS, LD = pd::LD;
  constexpr int64_t BLK = Stored<ST, MS>::BLK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* M1 = reinterpret_cast<CT*>(smem_raw);
  CT* M2 = M1 + MS * LD;
  CT* colbuf = M2 + (Q >= 1 ? MS * LD : 0);
  using FT = FactorTables<K, NPGX, CT>;
  FT& ft = *reinterpret_cast<FT*>(smem_raw + ((sizeof(CT) * ((Q >= 1 ? 2 : 1) * MS * LD + MS) + 15) / 16) * 16);
  int* perm = reinterpret_cast<int*>(&ft + 1);
  int* sh = perm + MS;
  const int blk = blockIdx.x, slab = blockIdx.y;
  const CtaGroup gr{(int)threadIdx.x, NTH};
  build_factor_tables<K, NPGX>(g, T, bs, blk, ft, gr);
  if (threadIdx.x == 0) { sh[0] = 0; sh[1] = 0; }
  __syncthreads();
  const bool conv = ph.conv != 0.0;
  ST* F = factors + ((int64_t)blk * g.N + slab) * (Q + 1) * (Q + 1) * BLK;
  bool ok;
  if constexpr (Q == 0) {
    assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M1, 0, 0, false, gr);
    __syncthreads();
    if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M1, 0, 0, gr);
    ok = invert_block<MS, LD, NTH>(M1, colbuf, perm, sh);
    store_colmajor<MS, LD, NTH>(M1, F);
  } else if constexpr (Q >= 2) {
    // left-looking block LU over the NT temporal sub-blocks (see block_op): the earlier
    // C_km and X_mj are read back from this block's own stored factors
    constexpr int NT = Q + 1;
    auto assemble = [&](CT* M, int a, int b) {
      assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M, a, b, false, gr);
      __syncthreads();
      if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M, a, b, gr);
      __syncthreads();
    };
    ok = true;
    for (int k = 0; k < NT; ++k) {
      assemble(M1, k, k);
      for (int m = 0; m < k; ++m)
        gemm_sub_stored<MS, LD, NTH>(M1, F + pos_low<NT>(k, m) * BLK, F + pos_up<NT>(m, k) * BLK);
      ok = invert_block<MS, LD, NTH>(M1, colbuf, perm, sh) && ok;
      store_colmajor<MS, LD, NTH>(M1, F + pos_diag<NT>(k) * BLK);
      __syncthreads();
      for (int j = k + 1; j < NT; ++j) {
        assemble(M2, k, j);
        for (int m = 0; m < k; ++m)
          gemm_sub_stored<MS, LD, NTH>(M2, F + pos_low<NT>(k, m) * BLK, F + pos_up<NT>(m, j) * BLK);
        gemm_block<MS, LD, NTH, CT>(M1, M2, CT(1));
        store_colmajor<MS, LD, NTH>(M2, F + pos_up<NT>(k, j) * BLK);
        __syncthreads();  // M2 is reassembled next; the stored block is read back later
      }
      for (int i = k + 1; i < NT; ++i) {
        assemble(M2, i, k);
        for (int m = 0; m < k; ++m)
          gemm_sub_stored<MS, LD, NTH>(M2, F + pos_low<NT>(i, m) * BLK, F + pos_up<NT>(m, k) * BLK);
        store_colmajor<MS, LD, NTH>(M2, F + pos_low<NT>(i, k) * BLK);
        __syncthreads();
      }
    }
  } else {
    // A00^{-1}
    assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M1, 0, 0, false, gr);
    __syncthreads();
    if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M1, 0, 0, gr);
    ok = invert_block<MS, LD, NTH>(M1, colbuf, perm, sh);
    store_colmajor<MS, LD, NTH>(M1, F);
    // X = A00^{-1} A01
    assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M2, 0, 1, false, gr);
    __syncthreads();
    if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M2, 0, 1, gr);
    gemm_block<MS, LD, NTH, CT>(M1, M2, CT(1));
    store_colmajor<MS, LD, NTH>(M2, F + 3 * BLK);
    // A10 (FP64 patch blocks: by the segments of its sparsity pattern)
    assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M1, 1, 0, false, gr);
    __syncthreads();
    if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M1, 1, 0, gr);
    if constexpr (sizeof(ST) == 8 && NPGX == 2 * K - 1) {
      if (bs.kind == 0) store_sparse_a10<K, MS, LD, NTH>(M1, F + 1 * BLK);
      else store_colmajor<MS, LD, NTH>(M1, F + 1 * BLK);
    } else {
      store_colmajor<MS, LD, NTH>(M1, F + 1 * BLK);
    }
    // S = A11 - A10 X
    gemm_block<MS, LD, NTH, CT>(M1, M2, CT(-1));
    assemble_const<K, Q, CT, LD, NPGX>(g, T, ph, ft, M2, 1, 1, true, gr);
    __syncthreads();
    if (conv) assemble_conv<K, Q, CT, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, ft, M2, 1, 1, gr);
    ok = invert_block<MS, LD, NTH>(M2, colbuf, perm, sh) && ok;
    store_colmajor<MS, LD, NTH>(M2, F + 2 * BLK);
  }
  if (!ok && threadIdx.x == 0) atomicExch(status, 1);
}

// Q2/Q1 DG(0) blocks (51 x 51) of the reduced-precision forms: one warp per
// (patch, slab), WPB warps per CTA, no barrier wider than a warp.  The warp builds
// its tables and assembles its block in FP32 in its own shared-memory tile (the
// same assembly as the CTA kernel, lane-strided), then inverts it in registers by
// the Gauss-Jordan elimination of gauss_jordan_reg (no row moves; pivot = largest
// |.| among the rows not yet used, compared to 16 mantissa bits, lowest row on ties): lane l holds rows l and
// l + 32.  Each step eliminates the current first column and appends the new
// column of the inverse at the end (every row shifts left by one), so the pivot
// column is always register 0, the column loop unrolls with constant register
// indices and the step loop stays rolled.  After MS steps a row holds the row of
// X with its columns in step order; the pivot order is undone in the column-major
// store: inv(A)[step of row i][pivot row of step j] = X[i][j].
template <typename ST>
struct FactorWarpSmem {
  static constexpr int MS = PD<1, 1>::MS, LD = PD<1, 1>::LD;
  float M[MS * LD];
  FactorTables<1, 1, float> ft;
  int prow[MS];
};

template <typename ST, int WPB>
__global__ void __launch_bounds__(32 * WPB)
block_factor_warp_kernel(LevelGeom g, FeTables T, PhysParams ph, BlockSet bs, const float* __restrict__ Ce,
                         ST* __restrict__ factors, int* __restrict__ status) {
  constexpr int K = 1, Q = 0, NPGX = 1;
  using SM = FactorWarpSmem<ST>;
  constexpr int MS = SM::MS, LD = SM::LD;
  static_assert(MS > 32 && MS <= 64, "two rows per lane");
  using SL = Stored<ST, MS>;
  constexpr int64_t BLK = SL::BLK;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  SM& sm = reinterpret_cast<SM*>(smem_raw)[w];
  const int nblk = g.npatch();
  const int64_t item = (int64_t)blockIdx.x * WPB + w;  // slab-major: neighbouring warps share cells
  if (item >= (int64_t)nblk * g.N) return;             // the whole warp leaves
  const int blk = (int)(item % nblk), slab = (int)(item / nblk);
  const WarpGroup gr{lane, 32};
  build_factor_tables<K, NPGX>(g, T, bs, blk, sm.ft, gr);
  __syncwarp();
  assemble_const<K, Q, float, LD, NPGX>(g, T, ph, sm.ft, sm.M, 0, 0, false, gr);
  __syncwarp();
  if (ph.conv != 0.0) assemble_conv<K, Q, float, LD, NPGX>(g, T, ph, bs, Ce, blk, slab, sm.ft, sm.M, 0, 0, gr);
  __syncwarp();
  const bool two = lane + 32 < MS;
  float a0[MS], a1[MS];
#pragma unroll
  for (int j = 0; j < MS; ++j) {
    a0[j] = sm.M[lane * LD + j];
    a1[j] = two ? sm.M[(lane + 32) * LD + j] : 0.f;
  }
  unsigned used = two ? 0u : 2u;  // bit 0: row lane, bit 1: row lane + 32 (absent rows count as used)
  int step0 = 0, step1 = 0;
  bool zero = false;
#pragma unroll 1
  for (int p = 0; p < MS; ++p) {
    // pivot: one integer max over keys that hold |x| to 16 mantissa bits above 127 - row
    // (rows already used have key 0)
    const unsigned k0 = (used & 1u) ? 0u : ((abs_key(a0[0]) & 0x7fffff80u) | (unsigned)(127 - lane));
    const unsigned k1 = (used & 2u) ? 0u : ((abs_key(a1[0]) & 0x7fffff80u) | (unsigned)(95 - lane));
    const int bi = 127 - (int)(__reduce_max_sync(FULL, max(k0, k1)) & 127u);
    const int owner = bi & 31;
    const bool hi = bi >= 32;
    const bool r0 = !hi && lane == owner, r1 = hi && lane == owner;
    const float pv = __shfl_sync(FULL, hi ? a1[0] : a0[0], owner);
    zero |= !(fabsf(pv) > 0.f);
    const float inv = 1.f / pv;
    // the pivot row keeps its entries (zero multiplier) and is scaled by its owner below
    const float f0 = r0 ? 0.f : a0[0], f1 = r1 ? 0.f : a1[0];
#pragma unroll
    for (int j = 1; j < MS; ++j) {
      const float rj = __shfl_sync(FULL, hi ? a1[j] : a0[j], owner) * inv;
      a0[j - 1] = fmaf(-f0, rj, a0[j]);
      a1[j - 1] = fmaf(-f1, rj, a1[j]);
    }
    a0[MS - 1] = r0 ? inv : -f0 * inv;
    a1[MS - 1] = r1 ? inv : -f1 * inv;
    if (r0) {
#pragma unroll
      for (int j = 0; j < MS - 1; ++j) a0[j] *= inv;
      used |= 1u;
      step0 = p;
    }
    if (r1) {
#pragma unroll
      for (int j = 0; j < MS - 1; ++j) a1[j] *= inv;
      used |= 2u;
      step1 = p;
    }
    if (lane == 0) sm.prow[p] = bi;
  }
  __syncwarp();
  ST* F = factors + ((int64_t)blk * g.N + slab) * BLK;
#pragma unroll
  for (int j = 0; j < MS; ++j) {
    const int col = sm.prow[j];
    narrow(a0[j], F[SL::at(step0, col)]);
    if (two) narrow(a1[j], F[SL::at(step1, col)]);
  }
  if (zero && lane == 0) atomicExch(status, 1);
}

// ---------------------------------------------------------------- smoother apply
// Persistent, warp-specialised.  CTA c owns patches c, c + gridDim.x, ...  A
// patch's stored factors are one contiguous run of N (q+1)^2 column-major blocks
// in the order they are consumed.  A producer warp streams them, in chunks of CC
// columns, into a ring of NS shared-memory slots with cp.async.bulk; slot s has a
// "full" mbarrier (transaction count = the chunk's bytes) and an "empty"
// mbarrier on which every consumer warp arrives once it has read the chunk, so
// the producer refills a slot as soon as it is free and about NS chunks stay in
// flight.  Consumer thread (i, g) multiplies row i by the g-th sub-range of each
// chunk's columns (G groups: 95-99% of the lanes issue FP64 FMAs, which bind on
// GB300) with one accumulator (FP64) or four (FP32/BF16); partial sums are combined in a fixed
// order after a named barrier of the consumer warps.  The next slab's right-hand
// side is prefetched into registers while the current slab's blocks are applied.
// Every wait is bounded: on timeout the kernel sets *err, drains its own copies
// in flight (bounded) and returns.
// Arithmetic type of the apply for each factor storage type: BF16 factors are
// widened to FP32 on load.
template <typename FT> struct ComputeType { using type = FT; };
template <> struct ComputeType<__nv_bfloat16> { using type = float; };
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }

// Tile variants of the smoother apply (chosen per level by the autotuner): column
// groups per chunk G, CTAs per SM and the shared-memory ring that streams the
// factor chunks.  Variants of one K with the same G sum in the same order.
//   Q2/Q1 (K = 1): G = 5 with 1, 4 or 3 CTAs per SM (176 / 43 / 64 KB rings);
//   Q3/Q2 (K = 2): G = 4 with one 480-thread CTA per SM (176 KB), or G = 2 with
//                  two or three 256-thread CTAs per SM (96 / 64 KB).
// The coarse 3x3 block (NPGX != 2K - 1) always takes variant 0.
constexpr int kApplyVariants = 5;  // tiles 0-2: CTA per block; 3: warp per block; 4: warp per block, bulk copies
// without tuning: three 64 KB CTAs per SM for Q2/Q1, one 480-thread CTA for Q3/Q2
inline int default_apply_variant(int k) { return k == 1 ? 2 : 0; }
template <int K, int V>
struct ApplyTile {
  static constexpr int G = K == 1 ? 5 : (V == 0 ? 4 : 2);
  // Q2/Q1 tile 1: four CTAs per SM with a two-block FP64 ring (47 KB each), so that
  // three other CTAs' GEMVs keep the FP64 pipe busy while one is in its serial phases
  // (jump coupling, group reduction)
  static constexpr int MINB = (K == 1 && V == 1) ? 4 : V + 1;
  static constexpr int RING_KB = V == 0 ? 176 : V == 1 ? (K == 1 ? 43 : 96) : 64;
};

template <int K, int Q, typename FT, int NPGX = 2 * K - 1, int V = 0>
struct ApplyCfg {
  using pd = PD<K, NPGX>;
  using CT = typename ComputeType<FT>::type;
  using TL = ApplyTile<K, NPGX == 2 * K - 1 ? V : 0>;
  static constexpr int MS = pd::MS, NT = Q + 1, NB = NT * NT;
  static constexpr int G = TL::G;                                 // column groups per chunk
  static constexpr int NCONS = (G * MS + 31) / 32 * 32;           // consumer threads
  static constexpr int NTH = NCONS + 32;                          // + one producer warp
  static constexpr int GR = 16 / (int)sizeof(FT);                 // elements per 16-byte granule
  using SL = Stored<FT, MS>;
  static constexpr int BLK = SL::BLK;                             // stored block elements
  static constexpr int BLK_BYTES = BLK * (int)sizeof(FT);
  // chunk width: whole block for k = 1; for k = 2, 28 columns (FP64, FP32) or 64 (BF16, whose
  // two-byte entries need twice the FMAs per byte: the wider chunk halves the per-chunk ring
  // work per FMA).  A multiple of GR columns keeps every chunk boundary on a 16-byte granule.
  static constexpr int CC = K == 1 ? (MS + GR - 1) / GR * GR : (sizeof(FT) == 2 ? 64 : (28 + GR - 1) / GR * GR);
  static constexpr int NCH = (MS + CC - 1) / CC;                  // chunks per block
  // columns per group and chunk (whole 16-byte column groups for the FP32 / BF16 Q2/Q1 blocks)
  static constexpr int SUB = SL::GRP ? ((CC + G - 1) / G + SL::GV - 1) / SL::GV * SL::GV : (CC + G - 1) / G;
  static constexpr int MSX = (MS + 3) / 4 * 4;                    // 16-byte rows of rhs / y in shared memory
  // four-wide loads of the input vector when every group's first column is 16-byte aligned
  static constexpr bool XV = sizeof(CT) == 4 && SUB % 4 == 0 && CC % 4 == 0;
  static constexpr int LAST = BLK - (NCH - 1) * CC * MS;          // last chunk carries the padding
  static constexpr int SLOT = CC * MS > LAST ? CC * MS : LAST;
  static constexpr int SLOT_ELEMS = (SLOT + GR - 1) / GR * GR;
  static constexpr int MINB = TL::MINB;                           // CTAs per SM
  static constexpr int RING_BYTES = TL::RING_KB * 1024;
  static constexpr int NS = RING_BYTES / (SLOT_ELEMS * (int)sizeof(FT)) < 16
                                ? RING_BYTES / (SLOT_ELEMS * (int)sizeof(FT))
                                : 16;
  static_assert((CC * MS * (int)sizeof(FT)) % 16 == 0, "chunk boundary off the 16-byte granule");
  static_assert(!SL::GRP || NCH == 1, "group-stored blocks stream as one chunk");
  static_assert(NS >= 2, "ring too small");
  // FP64 DG(1) patch blocks store A10 by segments (SpA10): its chunks hold IPC items of
  // every segment, NCH_SP of them per block
  static constexpr bool SPA = sizeof(FT) == 8 && Q == 1 && NPGX == 2 * K - 1;
  using SP = SpA10<K>;
  static constexpr int IPC = SPA ? SLOT_ELEMS / SP::NSEGP : 1;
  static constexpr int NCH_SP = SPA ? (SP::L + IPC - 1) / IPC : 1;
  static_assert(!SPA || (IPC >= 1 && SP::NSEGP <= NCONS && SP::ELEMS <= BLK && SP::MS == MS &&
                          SP::NSEGP <= G * MS),
                "A10 segments do not fit the tile");
};

template <int K, int Q, typename FT, int NPGX = 2 * K - 1, int V = 0>
struct ApplySmem {
  using C = ApplyCfg<K, Q, FT, NPGX, V>;
  using pd = PD<K, NPGX>;
  using CT = typename C::CT;
  unsigned long long full[C::NS];
  unsigned long long empty[C::NS];
  int abort_flag;  // written by any warp at any time
  int decision;    // abort decision of the consumers, published by consumer thread 0 before a barrier
  int issued;
  int sidx[C::MS];
  // the columns of real (non-padding) slots, in order, and where each chunk's start in
  // that list; dense = 1 when the block has no padding slot
  int cols[C::MS];
  int cst[C::NCH + 1];
  int dense;
  alignas(16) CT rhs[C::NT][C::MSX];
  alignas(16) CT y[C::NT][C::MSX];
  CT red[C::G][C::MS];  // group sums of a dense block; segment sums of a sparse A10 block
  CT yp[2][pd::NVG2];
  CT tm[2][pd::NVG2];
  CT mx[pd::NVG][pd::NVG];
  CT my[pd::NVG][pd::NVG];
};

// Every wait of the apply kernels is bounded in time: after kWaitLimitNs of the
// global nanosecond timer (checked every 256 polls) the wait gives up, the
// kernel raises the error flag, drains its own copies in flight and returns.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
  }
}
template <int NCONS>
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NCONS) : "memory");
}

// One unit of work of the smoother apply: block `blk` of a level, with that
// level's geometry, stored factors, right-hand side and output.
template <typename FT>
struct ApplyItem {
  LevelGeom g;
  BlockSet bs;
  const FT* factors;
  const double* r;
  double* out;  // patch outputs [slab][blk][a][slot] (kind 0) or the global solution (kind 1)
  int blk;
  // kind 0 only: patch outputs of the slab before this item's first slab (the
  // jump state when the slabs are processed in windows), or null (zero state)
  const double* prev;
  int fN, s0;  // the factor array's slabs per block and this item's first slab in it (g.N slabs from s0)
};

template <int K, int Q, typename FT, int NPGX, int V, class Items>
__device__ __forceinline__ void apply_persistent(const FeTables& T, const Items& items, int64_t nitems,
                                                 int* __restrict__ err) {
  using C = ApplyCfg<K, Q, FT, NPGX, V>;
  using pd = PD<K, NPGX>;
  using CT = typename C::CT;
  constexpr int MS = C::MS, NT = C::NT, NB = C::NB, NS = C::NS, NVG = pd::NVG, NCH = C::NCH, NCONS = C::NCONS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FT* ring = reinterpret_cast<FT*>(smem_raw);
  ApplySmem<K, Q, FT, NPGX, V>& sm =
      *reinterpret_cast<ApplySmem<K, Q, FT, NPGX, V>*>(smem_raw + (size_t)NS * C::SLOT_ELEMS * sizeof(FT));
  volatile int* abort_flag = &sm.abort_flag;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(smem_u32(&sm.full[i]), 1);
      mbar_init(smem_u32(&sm.empty[i]), NCONS / 32);
    }
    sm.abort_flag = 0;
    sm.decision = 0;
    sm.issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= NCONS) {  // ---------------- producer warp: walks the CTA's items and streams their chunks
    if (lane == 0) {
      int64_t s = 0;
      bool stop = false;
      for (int64_t it = blockIdx.x; it < nitems && !stop; it += gridDim.x) {
        const ApplyItem<FT> v = items(it);
        const bool sp = C::SPA && v.bs.kind == 0;
        const int64_t nblk = (int64_t)v.g.N * NB;
        for (int64_t bi = 0; bi < nblk && !stop; ++bi) {  // block index within the item
          const bool spb = sp && bi % NB == 1;  // the A10 block, stored by segments
          const int nch = spb ? C::NCH_SP : NCH;
          for (int k = 0; k < nch; ++k, ++s) {
            const int slot = (int)(s % NS);
            const int64_t u = s / NS;
            if (u > 0 && !mbar_wait_bounded(smem_u32(&sm.empty[slot]), (uint32_t)((u - 1) & 1))) {
              *abort_flag = 1;
              atomicExch(err, 1);
              stop = true;
              break;
            }
            if (*abort_flag) {
              stop = true;
              break;
            }
            const int64_t base = (((int64_t)v.blk * v.fN + v.s0) * NB + bi) * C::BLK;
            int64_t off;
            int elems;
            if (spb) {
              off = base + (int64_t)k * C::IPC * C::SP::NSEGP;
              elems = (min(C::SP::L, (k + 1) * C::IPC) - k * C::IPC) * C::SP::NSEGP;
            } else {
              off = base + (int64_t)k * C::CC * MS;
              elems = (k == NCH - 1) ? C::BLK - k * C::CC * MS : C::CC * MS;
            }
            const uint32_t bar = smem_u32(&sm.full[slot]);
            const uint32_t bytes = (uint32_t)(elems * sizeof(FT));
            mbar_expect_tx(bar, bytes);
            bulk_g2s(smem_u32(ring + (size_t)slot * C::SLOT_ELEMS), v.factors + off, bytes, bar);
            *(volatile int*)&sm.issued = (int)(s + 1 < 0x7fffffff ? s + 1 : 0x7fffffff);
          }
        }
      }
    }
    return;
  }

  // ---------------- consumer warps
  int cslot = 0;          // ring slot of the next chunk to consume
  uint32_t cphase = 0u;   // its mbarrier phase parity
  const bool gemv_thread = tid < C::G * MS;
  const int row = tid % MS, grp = tid / MS;
  bool aborted = false;
  for (int64_t it = blockIdx.x; it < nitems && !aborted; it += gridDim.x) {
    const ApplyItem<FT> v = items(it);
    const LevelGeom& g = v.g;
    const BlockSet& bs = v.bs;
    const double* __restrict__ r = v.r;
    double* __restrict__ out = v.out;
    const int blk = v.blk;
    const int nvg = bs.nvg, nv2g = nvg * nvg;
    int vx0, vy0, px0, py0;
    block_origin(g, bs, blk, vx0, vy0, px0, py0);
    for (int s = tid; s < MS; s += NCONS) sm.sidx[s] = decode_slot(g, bs, blk, s).sp;
    int cx0, cx1, cy0, cy1;
    own_cells(g, bs, vx0, cx0, cx1);
    own_cells(g, bs, vy0, cy0, cy1);
    for (int e = tid; e < NVG * NVG; e += NCONS) {
      const int i = e / NVG, j = e % NVG;
      const int xi = vx0 + i, xj = vx0 + j, yi = vy0 + i, yj = vy0 + j;
      const bool okx = i < nvg && j < nvg && xi >= 1 && xi <= g.nv - 2 && xj >= 1 && xj <= g.nv - 2;
      const bool oky = i < nvg && j < nvg && yi >= 1 && yi <= g.nv - 2 && yj >= 1 && yj <= g.nv - 2;
      sm.mx[i][j] = okx ? (CT)(g.h * vv1<K>(T.m1, g.n, xi, xj, cx0, cx1)) : (CT)0;
      sm.my[i][j] = oky ? (CT)(g.h * vv1<K>(T.m1, g.n, yi, yj, cy0, cy1)) : (CT)0;
    }
    for (int e = tid; e < 2 * pd::NVG2; e += NCONS) {
      const int c = e / pd::NVG2, tt = e % pd::NVG2;
      sm.yp[c][tt] = (v.prev && bs.kind == 0 && tt < nv2g)
                         ? (CT)v.prev[((int64_t)blk * NT + NT - 1) * MS + c * nv2g + tt]
                         : (CT)0;
    }
    consumer_sync<NCONS>();
    // Padding slots (off the domain, Dirichlet, the coarse block's pinned pressure) hold
    // zero in every block's input vector, so their columns contribute nothing: blocks of
    // boundary patches skip them (the output rows of padding slots stay zero).
    if (tid == 0) {
      int n = 0;
      for (int k = 0; k < NCH; ++k) {
        sm.cst[k] = n;
        for (int c = k * C::CC; c < min(MS, (k + 1) * C::CC); ++c)
          if (sm.sidx[c] >= 0) sm.cols[n++] = c;
      }
      sm.cst[NCH] = n;
      sm.dense = n == MS;
    }
    consumer_sync<NCONS>();
    // The column skip saves FP64 pipe time.  FP32 and BF16 blocks take the dense loop on
    // every patch: their padding columns multiply zero inputs (finite factor entries:
    // padding slots carry the identity), and the dense loop's four-wide input loads and
    // four accumulators issue far fewer instructions per FMA than the column list.
    const bool dense = sizeof(CT) == 4 || sm.dense != 0;
    // (a) gather of slab 0; later slabs come from the register prefetch
    for (int e = tid; e < NT * MS; e += NCONS) {
      const int a = e / MS, s = e % MS, sp = sm.sidx[s];
      sm.rhs[a][s] = sp >= 0 ? (CT)r[(int64_t)a * g.S + sp] : (CT)0;
    }
    const bool carry = v.prev != nullptr && bs.kind == 0;  // jump state from before the window
    const bool sparse = C::SPA && bs.kind == 0;             // A10 stored by segments
    for (int slab = 0; slab < g.N && !aborted; ++slab) {
      if (slab > 0 || carry) {
        // jump coupling: rhs_a += tau_a(0) M_u y_{n-1, last} (tensor-product mass on the slot grid)
        consumer_sync<NCONS>();
        for (int e = tid; e < 2 * nv2g; e += NCONS) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, jx = tt % nvg;
          CT acc = 0;
          for (int jy = 0; jy < nvg; ++jy) acc = fma(sm.my[iy][jy], sm.yp[c][jy * nvg + jx], acc);
          sm.tm[c][tt] = acc;
        }
        consumer_sync<NCONS>();
        for (int e = tid; e < 2 * nv2g; e += NCONS) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, ix = tt % nvg;
          CT acc = 0;
          for (int jx = 0; jx < nvg; ++jx) acc = fma(sm.mx[ix][jx], sm.tm[c][iy * nvg + jx], acc);
          const int s = c * nv2g + tt;
          if (sm.sidx[s] >= 0)
            for (int a = 0; a < NT; ++a) sm.rhs[a][s] += (CT)T.tau0[a] * acc;
        }
      }
      consumer_sync<NCONS>();
      // register prefetch of the next slab's right-hand side
      CT pf = 0;
      if (tid < NT * MS && slab + 1 < g.N) {
        const int sp = sm.sidx[tid % MS];
        if (sp >= 0) pf = (CT)r[((int64_t)(slab + 1) * NT + tid / MS) * g.S + sp];
      }
      // (c) the slab's stored blocks in block_op order (Q = 0: y0 = A^{-1} r0;  Q = 1:
      //     z0 = A00^{-1} r0, s1 = r1 - A10 z0, y1 = S^{-1} s1, y0 = z0 - X y1)
      for (int b = 0; b < NB; ++b) {
        const BlockOp op = block_op<NT>(b);
        const CT* xv = op.src_y ? sm.y[op.src] : sm.rhs[op.src];
        const bool spb = sparse && b == 1;
        CT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int k = 0; k < (spb ? C::NCH_SP : NCH); ++k) {
          const int slot = cslot;
          const bool ok = !aborted && mbar_wait_bounded(smem_u32(&sm.full[slot]), cphase);
          if (!ok) {
            aborted = true;
            *abort_flag = 1;
          }
          if (ok && spb) {
            if constexpr (C::SPA) {
              if (tid < C::SP::NSEGP) {
                // A10 by segments: this thread's segment, the chunk's items k IPC ..
                const FT* A = ring + (size_t)slot * C::SLOT_ELEMS;
                const short* cl = sp_tab<K>().col + tid;  // column of item i at cl[i NSEGP]
                const int i0 = k * C::IPC, i1 = min(C::SP::L, i0 + C::IPC);
#pragma unroll 4
                for (int i = i0; i < i1; ++i)
                  a0 = fma(widen(A[(i - i0) * C::SP::NSEGP + tid]), xv[__ldg(cl + i * C::SP::NSEGP)], a0);
              }
            }
          } else if (ok && gemv_thread && !dense) {
            // the chunk's real columns, split evenly over the G column groups
            const FT* A = ring + (size_t)slot * C::SLOT_ELEMS;
            const CT* xk = xv + k * C::CC;
            const int t0 = sm.cst[k], cnt = sm.cst[k + 1] - t0, sub = (cnt + C::G - 1) / C::G;
            const int tb = t0 + grp * sub, te = min(t0 + cnt, tb + sub);
#pragma unroll 4
            for (int t = tb; t < te; ++t) {
              const int c = sm.cols[t] - k * C::CC;
              a0 = fma(widen(A[C::SL::at(row, c)]), xk[c], a0);
            }
          } else if (ok && gemv_thread) {
            const FT* A = ring + (size_t)slot * C::SLOT_ELEMS;
            const int c0 = grp * C::SUB;
            const int ncol = min(C::CC, MS - k * C::CC);
            const int c1 = min(ncol, c0 + C::SUB);
            const CT* xk = xv + k * C::CC;
            int c = c0;
            if constexpr (sizeof(CT) == 8) {
              // FP64: the SM's FP64 pipe (2 FMA/clk on GB300) bounds the GEMV, not the
              // dependency chain of one thread, so a single accumulator spares the
              // three combining additions per block
#pragma unroll 4
              for (; c < c1; ++c) a0 = fma(widen(A[c * MS + row]), xk[c], a0);
            } else if constexpr (C::SL::GRP) {
              // Q2/Q1 FP32 / BF16: one 16-byte load holds this row's entries of a group of
              // GV columns; columns c0 + 4i + j accumulate in a_j, the column-major tail in a0
              constexpr int GV = C::SL::GV;
              const int cg = min(c1, C::SL::CG);
              const uint4* Ao = reinterpret_cast<const uint4*>(A + ((c / GV) * MS + row) * GV);
              for (; c < cg; c += GV, Ao += MS) {
                const uint4 w = *Ao;
                const float4 xa = *reinterpret_cast<const float4*>(xk + c);
                if constexpr (GV == 8) {
                  const float4 xb = *reinterpret_cast<const float4*>(xk + c + 4);
                  a0 = fma(bf16_lo(w.x), xa.x, a0);
                  a1 = fma(bf16_hi(w.x), xa.y, a1);
                  a2 = fma(bf16_lo(w.y), xa.z, a2);
                  a3 = fma(bf16_hi(w.y), xa.w, a3);
                  a0 = fma(bf16_lo(w.z), xb.x, a0);
                  a1 = fma(bf16_hi(w.z), xb.y, a1);
                  a2 = fma(bf16_lo(w.w), xb.z, a2);
                  a3 = fma(bf16_hi(w.w), xb.w, a3);
                } else {
                  a0 = fma(__uint_as_float(w.x), xa.x, a0);
                  a1 = fma(__uint_as_float(w.y), xa.y, a1);
                  a2 = fma(__uint_as_float(w.z), xa.z, a2);
                  a3 = fma(__uint_as_float(w.w), xa.w, a3);
                }
              }
              for (c = max(c, C::SL::CG); c < c1; ++c) a0 = fma(widen(A[C::SL::at(row, c)]), xk[c], a0);
            } else {
              // columns c0 + 4i + j accumulate in a_j, the tail in a0; the column pointer
              // steps by four columns, so the four loads take fixed offsets
              const FT* Ac = A + c * MS + row;
              for (; c + 3 < c1; c += 4, Ac += 4 * MS) {
                CT x0, x1, x2, x3;
                if constexpr (C::XV) {
                  const float4 xq = *reinterpret_cast<const float4*>(xk + c);
                  x0 = xq.x; x1 = xq.y; x2 = xq.z; x3 = xq.w;
                } else {
                  x0 = xk[c]; x1 = xk[c + 1]; x2 = xk[c + 2]; x3 = xk[c + 3];
                }
                a0 = fma(widen(Ac[0]), x0, a0);
                a1 = fma(widen(Ac[MS]), x1, a1);
                a2 = fma(widen(Ac[2 * MS]), x2, a2);
                a3 = fma(widen(Ac[3 * MS]), x3, a3);
              }
              for (; c < c1; ++c, Ac += MS) a0 = fma(widen(Ac[0]), xk[c], a0);
            }
          }
          __syncwarp();
          if (ok && lane == 0) mbar_arrive(smem_u32(&sm.empty[slot]));  // this warp is done with the slot
          if (++cslot == NS) {
            cslot = 0;
            cphase ^= 1u;
          }
        }
        if (spb) {
          if constexpr (C::SPA)
            if (tid < C::SP::NSEGP) (&sm.red[0][0])[tid] = a0;
        } else if (gemv_thread) {
          sm.red[grp][row] = sizeof(CT) == 8 ? a0 : (a0 + a1) + (a2 + a3);
        }
        if (tid == 0) sm.decision = *abort_flag;  // one reader, so every consumer decides alike
        consumer_sync<NCONS>();
        if (sm.decision) {
          aborted = true;
          break;
        }
        if (tid < MS) {
          CT sum = CT(0);
          if constexpr (C::SPA) {
            if (spb) {  // the row's segment sums in column order
              const SpTab<K>& tb = sp_tab<K>();
              const int j0 = __ldg(&tb.start[tid]), nj = __ldg(&tb.nseg[tid]);
              const CT* seg = &sm.red[0][0];
              sum = seg[j0];
              for (int j = 1; j < nj; ++j) sum += seg[j0 + j];
            }
          }
          if (!spb) {
            sum = sm.red[0][tid];
#pragma unroll
            for (int h = 1; h < C::G; ++h) sum += sm.red[h][tid];
          }
          if (op.dst == 0) sm.y[op.di][tid] = sum;
          else if (op.dst == 1) sm.rhs[op.di][tid] -= sum;
          else sm.y[op.di][tid] -= sum;
        }
        consumer_sync<NCONS>();
      }
      if (aborted) break;
      // output, jump state, next right-hand side
      for (int e = tid; e < NT * MS; e += NCONS) {
        const int a = e / MS, s = e % MS;
        if (bs.kind == 0) {
          out[(((int64_t)slab * g.npatch() + blk) * NT + a) * MS + s] = (double)sm.y[a][s];
        } else if (sm.sidx[s] >= 0) {
          out[((int64_t)slab * NT + a) * g.S + sm.sidx[s]] = (double)sm.y[a][s];
        }
      }
      for (int e = tid; e < 2 * nv2g; e += NCONS) {
        const int c = e / nv2g, tt = e % nv2g;
        sm.yp[c][tt] = sm.y[NT - 1][c * nv2g + tt];
      }
      if (tid < NT * MS) sm.rhs[tid / MS][tid % MS] = pf;
    }
    consumer_sync<NCONS>();
  }
  if (aborted && tid == 0) {
    // the last NS issued chunks are the latest copy into each slot
    const int64_t issued = *(volatile int*)&sm.issued;
    for (int64_t s = issued > NS ? issued - NS : 0; s < issued; ++s)
      mbar_wait_bounded(smem_u32(&sm.full[(int)(s % NS)]), (uint32_t)((s / NS) & 1));
    atomicExch(err, 1);
  }
}

// The blocks of one level, optionally split into chunks of Lc slabs (time-parallel
// solve): item it is chunk c_first + it / nblk of block it % nblk.  prev_mode 0: zero
// jump state; 1: chunk c starts from the state after chunk c - 1 (prev[c - 1], one
// [block][a][slot] slab of outputs per chunk; chunk 0 from zero); 2: every item
// starts from the same state prev.
template <typename FT>
struct SingleItems {
  LevelGeom g;
  BlockSet bs;
  const FT* factors;
  const double* r;
  double* out;
  const double* prev;
  int nblk = 1, nchunk = 1, Lc = 0, c_first = 0, prev_mode = 0;
  __device__ ApplyItem<FT> operator()(int64_t it) const {
    ApplyItem<FT> v;
    v.g = g;
    v.bs = bs;
    v.factors = factors;
    v.fN = g.N;
    if (nchunk == 1) {
      v.r = r;
      v.out = out;
      v.blk = (int)it;
      v.prev = prev;
      v.s0 = 0;
      return v;
    }
    const int c = c_first + (int)(it / nblk);
    v.blk = (int)(it % nblk);
    v.s0 = c * Lc;
    v.g.N = min(Lc, g.N - v.s0);
    const int64_t slab_out = (int64_t)g.npatch() * g.nt * bs.ms;
    v.r = r + (int64_t)v.s0 * g.nt * g.S;
    v.out = out + v.s0 * slab_out;
    v.prev = prev_mode == 1 ? (c > 0 ? prev + (int64_t)(c - 1) * slab_out : nullptr) : prev_mode == 2 ? prev : nullptr;
    return v;
  }
};

template <typename FT>
struct BatchItems {
  const BatchSeg* segs;
  int nseg;
  const double* r;   // arena of right-hand sides at this depth (kind 0)
  double* yp;        // patch-output arena (kind 0)
  bool coarse;       // kind 1: absolute per-member pointers xa / ya
  __device__ ApplyItem<FT> operator()(int64_t it) const {
    const int m = batch_find<BU_PATCH>(segs, nseg, it);
    const BatchSeg& sg = segs[m];
    ApplyItem<FT> v;
    v.g = sg.g;
    v.bs = sg.bs;
    v.factors = static_cast<const FT*>(sg.factors);
    v.blk = (int)(it - sg.u_patch);
    v.prev = nullptr;
    v.fN = sg.g.N;
    v.s0 = 0;
    if (coarse) {
      v.r = sg.xa;
      v.out = sg.ya;
    } else {
      v.r = r + sg.off;
      v.out = yp + sg.off_yp;
    }
    return v;
  }
};

// ---------------------------------------------------------------- warp-per-patch apply (tile 3)
// Each warp owns one item at a time: it streams the item's factor blocks straight
// from global memory (column-major blocks: for a column, the warp's lanes read
// consecutive rows, R rows per lane) and needs no block-wide barrier, only warp
// synchronisation between the phases of a slab.  The arithmetic per row is the
// CTA tile's with one group (G = 1): one running sum per row over all columns.
constexpr int kWarpTileWarps = 8;

template <int K, int Q, typename FT>
struct WarpSmem {
  using pd = PD<K>;
  using CT = typename ComputeType<FT>::type;
  static constexpr int MS = pd::MS, NT = Q + 1;
  // 16-byte rows where the octet loops load the input four-wide
  static constexpr bool GRP = Stored<FT, MS>::GRP;
  static constexpr int MSW = GRP ? (MS + 3) / 4 * 4 : MS;
  alignas(GRP ? 16 : alignof(CT)) CT rhs[NT][MSW];
  alignas(GRP ? 16 : alignof(CT)) CT y[NT][MSW];
  CT yp[2][pd::NVG2];
  CT tm[2][pd::NVG2];
  CT mx[pd::NVG][pd::NVG];
  CT my[pd::NVG][pd::NVG];
  int sidx[MS];
};

template <int K, int Q, typename FT, class Items>
__device__ __forceinline__ void warp_apply(const FeTables& T, const Items& items, int64_t nitems) {
  using pd = PD<K>;
  using CT = typename ComputeType<FT>::type;
  using C = ApplyCfg<K, Q, FT>;
  constexpr int MS = pd::MS, NT = Q + 1, NB = NT * NT, NVG = pd::NVG, R = (MS + 31) / 32;
  extern __shared__ __align__(16) unsigned char wsm_raw[];  // kWarpTileWarps WarpSmem (dynamic: > 48 KB for k = 2)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  WarpSmem<K, Q, FT>& sm = reinterpret_cast<WarpSmem<K, Q, FT>*>(wsm_raw)[w];
  const int64_t nwarps = (int64_t)gridDim.x * kWarpTileWarps;
  for (int64_t it = (int64_t)blockIdx.x * kWarpTileWarps + w; it < nitems; it += nwarps) {
    const ApplyItem<FT> v = items(it);
    const LevelGeom& g = v.g;
    const BlockSet& bs = v.bs;
    const int blk = v.blk, nvg = bs.nvg, nv2g = nvg * nvg;
    int vx0, vy0, px0, py0;
    block_origin(g, bs, blk, vx0, vy0, px0, py0);
    for (int s = lane; s < MS; s += 32) sm.sidx[s] = decode_slot(g, bs, blk, s).sp;
    int cx0, cx1, cy0, cy1;
    own_cells(g, bs, vx0, cx0, cx1);
    own_cells(g, bs, vy0, cy0, cy1);
    for (int e = lane; e < NVG * NVG; e += 32) {
      const int i = e / NVG, j = e % NVG;
      const int xi = vx0 + i, xj = vx0 + j, yi = vy0 + i, yj = vy0 + j;
      const bool okx = i < nvg && j < nvg && xi >= 1 && xi <= g.nv - 2 && xj >= 1 && xj <= g.nv - 2;
      const bool oky = i < nvg && j < nvg && yi >= 1 && yi <= g.nv - 2 && yj >= 1 && yj <= g.nv - 2;
      sm.mx[i][j] = okx ? (CT)(g.h * vv1<K>(T.m1, g.n, xi, xj, cx0, cx1)) : (CT)0;
      sm.my[i][j] = oky ? (CT)(g.h * vv1<K>(T.m1, g.n, yi, yj, cy0, cy1)) : (CT)0;
    }
    const bool carry = v.prev != nullptr;
    for (int e = lane; e < 2 * pd::NVG2; e += 32) {
      const int c = e / pd::NVG2, tt = e % pd::NVG2;
      sm.yp[c][tt] = (carry && tt < nv2g) ? (CT)v.prev[((int64_t)blk * NT + NT - 1) * MS + c * nv2g + tt] : (CT)0;
    }
    __syncwarp();
    for (int e = lane; e < NT * MS; e += 32) {
      const int a = e / MS, s = e % MS, sp = sm.sidx[s];
      sm.rhs[a][s] = sp >= 0 ? (CT)v.r[(int64_t)a * g.S + sp] : (CT)0;
    }
    for (int slab = 0; slab < g.N; ++slab) {
      __syncwarp();
      if (slab > 0 || carry) {
        for (int e = lane; e < 2 * nv2g; e += 32) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, jx = tt % nvg;
          CT acc = 0;
          for (int jy = 0; jy < nvg; ++jy) acc = fma(sm.my[iy][jy], sm.yp[c][jy * nvg + jx], acc);
          sm.tm[c][tt] = acc;
        }
        __syncwarp();
        for (int e = lane; e < 2 * nv2g; e += 32) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, ix = tt % nvg;
          CT acc = 0;
          for (int jx = 0; jx < nvg; ++jx) acc = fma(sm.mx[ix][jx], sm.tm[c][iy * nvg + jx], acc);
          const int s = c * nv2g + tt;
          if (sm.sidx[s] >= 0)
            for (int a = 0; a < NT; ++a) sm.rhs[a][s] += (CT)T.tau0[a] * acc;
        }
        __syncwarp();
      }
      // register prefetch of the next slab's right-hand side
      CT pf[(NT * MS + 31) / 32];
#pragma unroll
      for (int u = 0; u < (NT * MS + 31) / 32; ++u) {
        const int e = lane + 32 * u;
        pf[u] = 0;
        if (e < NT * MS && slab + 1 < g.N) {
          const int sp = sm.sidx[e % MS];
          if (sp >= 0) pf[u] = (CT)v.r[((int64_t)(slab + 1) * NT + e / MS) * g.S + sp];
        }
      }
      // the stored blocks in block_op order
      for (int b = 0; b < NB; ++b) {
        const BlockOp op = block_op<NT>(b);
        const CT* xv = op.src_y ? sm.y[op.src] : sm.rhs[op.src];
        const FT* A = v.factors + (((int64_t)blk * v.fN + v.s0 + slab) * NB + b) * C::BLK;
        CT acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        if constexpr (Stored<FT, MS>::GRP) {
          // one 16-byte load per row and group of columns, then the column-major tail;
          // even groups and the tail accumulate in acc, odd groups in acc2 (two chains)
          using SL = Stored<FT, MS>;
          static_assert(SL::CG / SL::GV % 2 == 0, "groups in pairs");
          CT acc2[R];
#pragma unroll
          for (int r = 0; r < R; ++r) acc2[r] = 0;
          for (int o = 0; o < SL::CG / SL::GV; o += 2) {
            float4 xa, xb, xc, xd;
            grp_x<FT>(xv + SL::GV * o, xa, xb);
            grp_x<FT>(xv + SL::GV * (o + 1), xc, xd);
            const uint4* Ao = reinterpret_cast<const uint4*>(A) + (int64_t)o * MS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int row = lane + 32 * r;
              if (row < MS) {
                acc[r] = grp_fma<FT>(__ldg(Ao + row), xa, xb, acc[r]);
                acc2[r] = grp_fma<FT>(__ldg(Ao + MS + row), xc, xd, acc2[r]);
              }
            }
          }
#pragma unroll
          for (int c = SL::CG; c < MS; ++c) {
            const CT xc = xv[c];
            const FT* col = A + SL::at(0, c);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int row = lane + 32 * r;
              if (row < MS) acc[r] = fma(widen(__ldg(col + row)), xc, acc[r]);
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] += acc2[r];
        } else {
#pragma unroll 4
          for (int c = 0; c < MS; ++c) {
            const CT xc = xv[c];
            const FT* col = A + (int64_t)c * MS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int row = lane + 32 * r;
              if (row < MS) acc[r] = fma(widen(__ldg(col + row)), xc, acc[r]);
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int row = lane + 32 * r;
          if (row >= MS) continue;
          if (op.dst == 0) sm.y[op.di][row] = acc[r];
          else if (op.dst == 1) sm.rhs[op.di][row] -= acc[r];
          else sm.y[op.di][row] -= acc[r];
        }
        __syncwarp();
      }
      for (int e = lane; e < NT * MS; e += 32) {
        const int a = e / MS, s = e % MS;
        if (bs.kind == 0) {
          v.out[(((int64_t)slab * g.npatch() + blk) * NT + a) * MS + s] = (double)sm.y[a][s];
        } else if (sm.sidx[s] >= 0) {
          v.out[((int64_t)slab * NT + a) * g.S + sm.sidx[s]] = (double)sm.y[a][s];
        }
      }
      for (int e = lane; e < 2 * nv2g; e += 32) {
        const int c = e / nv2g, tt = e % nv2g;
        sm.yp[c][tt] = sm.y[NT - 1][c * nv2g + tt];
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < (NT * MS + 31) / 32; ++u) {
        const int e = lane + 32 * u;
        if (e < NT * MS) sm.rhs[e / MS][e % MS] = pf[u];
      }
    }
    __syncwarp();
  }
}

template <int K, int Q, typename FT, int NPGX, int V>
__global__ void __launch_bounds__(ApplyCfg<K, Q, FT, NPGX, V>::NTH, ApplyCfg<K, Q, FT, NPGX, V>::MINB)
block_apply_kernel(LevelGeom g, FeTables T, SingleItems<FT> items, int64_t nitems, int* __restrict__ err) {
  apply_persistent<K, Q, FT, NPGX, V>(T, items, nitems, err);
}

template <int K, int Q, typename FT, int NPGX, int V>
__global__ void __launch_bounds__(ApplyCfg<K, Q, FT, NPGX, V>::NTH, ApplyCfg<K, Q, FT, NPGX, V>::MINB)
bt_block_apply_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t nitems, FeTables T,
                      const double* __restrict__ r, double* __restrict__ yp, int coarse, int* __restrict__ err) {
  apply_persistent<K, Q, FT, NPGX, V>(T, BatchItems<FT>{segs, nseg, r, yp, coarse != 0}, nitems, err);
}

template <int K, int Q, typename FT>
__global__ void __launch_bounds__(32 * kWarpTileWarps)
warp_apply_kernel(FeTables T, SingleItems<FT> items, int64_t nitems) {
  warp_apply<K, Q, FT>(T, items, nitems);
}

template <int K, int Q, typename FT>
__global__ void __launch_bounds__(32 * kWarpTileWarps)
bt_warp_apply_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t nitems, FeTables T,
                     const double* __restrict__ r, double* __restrict__ yp) {
  warp_apply<K, Q, FT>(T, BatchItems<FT>{segs, nseg, r, yp, false}, nitems);
}

// Tile 4 (Q2/Q1 DG(0) only): a warp per patch as in tile 3, with each slab's block
// (one contiguous column-major m x m block) brought into the warp's shared memory by
// a single bulk copy (cp.async.bulk completing on an mbarrier), two slabs ahead of
// its use.  Tile 3 keeps a few column loads in flight per warp and waits for them
// slab after slab; here a whole block is in flight while the one before it is
// applied.  The GEMV reads the block in the same order as tile 3 (bitwise the same
// result).  Every wait is bounded: on timeout the warp raises *err, waits (bounded)
// for its own copies still in flight and leaves.
constexpr int kWarpBulkWarps = 4;

template <typename FT>
struct alignas(16) WarpBulkSmem {
  static constexpr int MS = PD<1>::MS;
  static constexpr int BLK = Stored<FT, MS>::BLK;  // the stored block (a multiple of 16 bytes)
  FT buf[2][BLK];
  unsigned long long full[2];
  WarpSmem<1, 0, FT> w;
};

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename FT, class Items>
__device__ __forceinline__ void warp_apply_bulk(const FeTables& T, const Items& items, int64_t nitems,
                                                int* __restrict__ err) {
  constexpr int K = 1;
  using pd = PD<K>;
  using CT = typename ComputeType<FT>::type;
  using SB = WarpBulkSmem<FT>;
  constexpr int MS = pd::MS, NVG = pd::NVG, R = (MS + 31) / 32, RP = (MS + 31) / 32;
  constexpr uint32_t BYTES = (uint32_t)(SB::BLK * sizeof(FT));
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char wsm_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  SB& sb = reinterpret_cast<SB*>(wsm_raw)[w];
  WarpSmem<1, 0, FT>& sm = sb.w;
  if (lane == 0) {
    mbar_init(smem_u32(&sb.full[0]), 1);
    mbar_init(smem_u32(&sb.full[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // completed uses of each buffer (the parity of its next wait) and copies in flight, as
  // bit 0 (buffer 0) and bit 1 (buffer 1) -- scalars, so that nothing goes to local memory
  uint32_t used0 = 0u, used1 = 0u, pending = 0u;
  bool aborted = false;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpBulkWarps;
  for (int64_t it = (int64_t)blockIdx.x * kWarpBulkWarps + w; it < nitems && !aborted; it += nwarps) {
    const ApplyItem<FT> v = items(it);
    const LevelGeom& g = v.g;
    const BlockSet& bs = v.bs;
    const int blk = v.blk, nvg = bs.nvg, nv2g = nvg * nvg;
    const FT* fblk = v.factors + ((int64_t)blk * v.fN + v.s0) * SB::BLK;  // slab 0 of this item
    // copies of the first two slabs' blocks
    for (int sl = 0; sl < 2 && sl < g.N; ++sl) {
      if (lane == 0) {
        fence_proxy_async();
        const uint32_t bar = smem_u32(&sb.full[sl]);
        mbar_expect_tx(bar, BYTES);
        bulk_g2s(smem_u32(sb.buf[sl]), fblk + (int64_t)sl * SB::BLK, BYTES, bar);
      }
      pending |= 1u << sl;
    }
    int vx0, vy0, px0, py0;
    block_origin(g, bs, blk, vx0, vy0, px0, py0);
    for (int s = lane; s < MS; s += 32) sm.sidx[s] = decode_slot(g, bs, blk, s).sp;
    int cx0, cx1, cy0, cy1;
    own_cells(g, bs, vx0, cx0, cx1);
    own_cells(g, bs, vy0, cy0, cy1);
    for (int e = lane; e < NVG * NVG; e += 32) {
      const int i = e / NVG, j = e % NVG;
      const int xi = vx0 + i, xj = vx0 + j, yi = vy0 + i, yj = vy0 + j;
      const bool okx = i < nvg && j < nvg && xi >= 1 && xi <= g.nv - 2 && xj >= 1 && xj <= g.nv - 2;
      const bool oky = i < nvg && j < nvg && yi >= 1 && yi <= g.nv - 2 && yj >= 1 && yj <= g.nv - 2;
      sm.mx[i][j] = okx ? (CT)(g.h * vv1<K>(T.m1, g.n, xi, xj, cx0, cx1)) : (CT)0;
      sm.my[i][j] = oky ? (CT)(g.h * vv1<K>(T.m1, g.n, yi, yj, cy0, cy1)) : (CT)0;
    }
    const bool carry = v.prev != nullptr;
    for (int e = lane; e < 2 * pd::NVG2; e += 32) {
      const int c = e / pd::NVG2, tt = e % pd::NVG2;
      sm.yp[c][tt] = (carry && tt < nv2g) ? (CT)v.prev[(int64_t)blk * MS + c * nv2g + tt] : (CT)0;
    }
    __syncwarp();
    for (int s = lane; s < MS; s += 32) {
      const int sp = sm.sidx[s];
      sm.rhs[0][s] = sp >= 0 ? (CT)v.r[sp] : (CT)0;
    }
    // the right-hand sides are loaded into registers two slabs ahead of their use, so
    // that a load's latency is covered by a whole slab of work
    static_assert(RP == 2, "two right-hand-side entries per lane");
    const int sp0 = sm.sidx[lane], sp1 = lane + 32 < MS ? sm.sidx[lane + 32] : -1;
    CT pa = 0, pb = 0;  // slab + 1
    if (1 < g.N) {
      if (sp0 >= 0) pa = (CT)v.r[(int64_t)g.S + sp0];
      if (sp1 >= 0) pb = (CT)v.r[(int64_t)g.S + sp1];
    }
    for (int slab = 0; slab < g.N; ++slab) {
      const int b = slab & 1;
      __syncwarp();
      if (slab > 0 || carry) {
        for (int e = lane; e < 2 * nv2g; e += 32) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, jx = tt % nvg;
          CT acc = 0;
          for (int jy = 0; jy < nvg; ++jy) acc = fma(sm.my[iy][jy], sm.yp[c][jy * nvg + jx], acc);
          sm.tm[c][tt] = acc;
        }
        __syncwarp();
        for (int e = lane; e < 2 * nv2g; e += 32) {
          const int c = e / nv2g, tt = e % nv2g, iy = tt / nvg, ix = tt % nvg;
          CT acc = 0;
          for (int jx = 0; jx < nvg; ++jx) acc = fma(sm.mx[ix][jx], sm.tm[c][iy * nvg + jx], acc);
          const int s = c * nv2g + tt;
          if (sm.sidx[s] >= 0) sm.rhs[0][s] += (CT)T.tau0[0] * acc;
        }
        __syncwarp();
      }
      CT qa = 0, qb = 0;  // slab + 2
      if (slab + 2 < g.N) {
        if (sp0 >= 0) qa = (CT)v.r[(int64_t)(slab + 2) * g.S + sp0];
        if (sp1 >= 0) qb = (CT)v.r[(int64_t)(slab + 2) * g.S + sp1];
      }
      // this slab's block
      const bool got = mbar_wait_bounded(smem_u32(&sb.full[b]), (b ? used1 : used0) & 1u);
      if (!__all_sync(FULL, got)) {
        aborted = true;
        break;
      }
      if (b) ++used1;
      else ++used0;
      pending &= ~(1u << b);
      const FT* A = sb.buf[b];
      CT acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = 0;
      if constexpr (Stored<FT, MS>::GRP) {  // tile 3's loops and chains on the shared-memory copy
        using SL = Stored<FT, MS>;
        CT acc2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc2[r] = 0;
        for (int o = 0; o < SL::CG / SL::GV; o += 2) {
          float4 xa, xb, xc, xd;
          grp_x<FT>(&sm.rhs[0][SL::GV * o], xa, xb);
          grp_x<FT>(&sm.rhs[0][SL::GV * (o + 1)], xc, xd);
          const uint4* Ao = reinterpret_cast<const uint4*>(A) + o * MS;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = lane + 32 * r;
            if (row < MS) {
              acc[r] = grp_fma<FT>(Ao[row], xa, xb, acc[r]);
              acc2[r] = grp_fma<FT>(Ao[MS + row], xc, xd, acc2[r]);
            }
          }
        }
#pragma unroll
        for (int c = SL::CG; c < MS; ++c) {
          const CT xc = sm.rhs[0][c];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = lane + 32 * r;
            if (row < MS) acc[r] = fma(widen(A[SL::at(row, c)]), xc, acc[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += acc2[r];
      } else {
#pragma unroll 4
        for (int c = 0; c < MS; ++c) {
          const CT xc = sm.rhs[0][c];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = lane + 32 * r;
            if (row < MS) acc[r] = fma(widen(A[c * MS + row]), xc, acc[r]);
          }
        }
      }
      __syncwarp();
      if (slab + 2 < g.N) {  // the buffer is free again: the block two slabs ahead
        if (lane == 0) {
          fence_proxy_async();
          const uint32_t bar = smem_u32(&sb.full[b]);
          mbar_expect_tx(bar, BYTES);
          bulk_g2s(smem_u32(sb.buf[b]), fblk + (int64_t)(slab + 2) * SB::BLK, BYTES, bar);
        }
        pending |= 1u << b;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = lane + 32 * r;
        if (row < MS) sm.y[0][row] = acc[r];
      }
      __syncwarp();
      for (int s = lane; s < MS; s += 32) {
        if (bs.kind == 0) {
          v.out[((int64_t)slab * g.npatch() + blk) * MS + s] = (double)sm.y[0][s];
        } else if (sm.sidx[s] >= 0) {
          v.out[(int64_t)slab * g.S + sm.sidx[s]] = (double)sm.y[0][s];
        }
      }
      for (int e = lane; e < 2 * nv2g; e += 32) {
        const int c = e / nv2g, tt = e % nv2g;
        sm.yp[c][tt] = sm.y[0][c * nv2g + tt];
      }
      __syncwarp();
      sm.rhs[0][lane] = pa;
      if (lane + 32 < MS) sm.rhs[0][lane + 32] = pb;
      pa = qa;
      pb = qb;
    }
    __syncwarp();
  }
  if (aborted) {
    // this warp's copies still in flight land before it leaves (each wait bounded)
    if (lane == 0) {
      if (pending & 1u) mbar_wait_bounded(smem_u32(&sb.full[0]), used0 & 1u);
      if (pending & 2u) mbar_wait_bounded(smem_u32(&sb.full[1]), used1 & 1u);
      atomicExch(err, 1);
    }
  }
}

template <typename FT>
__global__ void __launch_bounds__(32 * kWarpBulkWarps)
warp_bulk_apply_kernel(FeTables T, SingleItems<FT> items, int64_t nitems, int* __restrict__ err) {
  warp_apply_bulk<FT>(T, items, nitems, err);
}

template <typename FT>
__global__ void __launch_bounds__(32 * kWarpBulkWarps)
bt_warp_bulk_apply_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t nitems, FeTables T,
                          const double* __restrict__ r, double* __restrict__ yp, int* __restrict__ err) {
  warp_apply_bulk<FT>(T, BatchItems<FT>{segs, nseg, r, yp, false}, nitems, err);
}

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceildiv(int a, int b) { return -floordiv(-a, b); }

template <int K, int Q>
__device__ __forceinline__ void scatter_body(const LevelGeom& g, const double* __restrict__ Yp,
                                             double* __restrict__ y, int64_t idx, int weighted) {
  using pd = PD<K>;
  constexpr int MS = pd::MS, NT = Q + 1;
  const int S = g.S, nv = g.nv, nv2 = nv * nv, n = g.n, np1 = n + 1;
  const int64_t blkt = idx / S;
  const int sp = int(idx % S);
  const int slab = int(blkt / NT), a = int(blkt % NT);
  double acc = 0.0;
  int cnt = 0;  // number of patches holding the DoF
  if (sp < 2 * nv2) {
    const int c = sp / nv2, t = sp % nv2, gx = t % nv, gy = t / nv;
    if (gx == 0 || gy == 0 || gx == nv - 1 || gy == nv - 1) { y[idx] = 0.0; return; }
    const int p = K + 1;
    const int I0 = max(0, ceildiv(gx, p) - 1), I1 = min(n, gx / p + 1);
    const int J0 = max(0, ceildiv(gy, p) - 1), J1 = min(n, gy / p + 1);
    for (int J = J0; J <= J1; ++J)
      for (int I = I0; I <= I1; ++I) {
        const int lx = gx - (I - 1) * p, ly = gy - (J - 1) * p;
        const int s = c * pd::NVG2 + ly * pd::NVG + lx;
        acc += Yp[(((int64_t)slab * np1 * np1 + J * np1 + I) * NT + a) * MS + s];
        ++cnt;
      }
  } else {
    const int t = sp - 2 * nv2, px = t % g.np, py = t / g.np;
    const int I0 = max(0, ceildiv(px - K + 1, K)), I1 = min(n, floordiv(px + K - 1, K));
    const int J0 = max(0, ceildiv(py - K + 1, K)), J1 = min(n, floordiv(py + K - 1, K));
    for (int J = J0; J <= J1; ++J)
      for (int I = I0; I <= I1; ++I) {
        const int lx = px - (I * K - (K - 1)), ly = py - (J * K - (K - 1));
        const int s = 2 * pd::NVG2 + ly * pd::NPG + lx;
        acc += Yp[(((int64_t)slab * np1 * np1 + J * np1 + I) * NT + a) * MS + s];
        ++cnt;
      }
  }
  y[idx] = (weighted && cnt > 0) ? acc / cnt : acc;
}

template <int K, int Q>
__global__ void scatter_kernel(LevelGeom g, const double* __restrict__ Yp, double* __restrict__ y, int weighted) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  scatter_body<K, Q>(g, Yp, y, idx, weighted);
}

template <int K, int Q>
__global__ void bt_scatter_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs,
                                  const double* __restrict__ yp, double* __restrict__ y) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const LevelGeom g = segs[m].g;
  scatter_body<K, Q>(g, yp + segs[m].off_yp, y + segs[m].off, u - segs[m].u_dof, segs[m].bs.weighted);
}

template <int K, int Q, typename CT, typename ST, int NPGX = 2 * K - 1>
void run_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const BlockSet& bs, const CT* Ce,
                ST* factors, int* status, cudaStream_t s) {
  using pd = PD<K, NPGX>;
  constexpr int NTH = K == 1 ? 256 : 512;
  const size_t mats = ((sizeof(CT) * ((Q >= 1 ? 2 : 1) * pd::MS * pd::LD + pd::MS) + 15) / 16) * 16;
  const size_t smem = mats + sizeof(FactorTables<K, NPGX, CT>) + sizeof(int) * (pd::MS + 2);
  auto kern = block_factor_kernel<K, Q, CT, ST, NTH, NPGX>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int nblk = bs.kind == 0 ? g.npatch() : 1;
  kern<<<dim3(nblk, g.N), NTH, smem, s>>>(g, T, ph, bs, Ce, factors, status);
  WR_LAUNCH_CHECK();
}

template <typename ST>
void run_factor_warp(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const BlockSet& bs, const float* Ce,
                     ST* factors, int* status, cudaStream_t s) {
  constexpr int WPB = 4;
  const size_t smem = sizeof(FactorWarpSmem<ST>) * WPB;
  auto kern = block_factor_warp_kernel<ST, WPB>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t items = (int64_t)g.npatch() * g.N;
  kern<<<(unsigned)((items + WPB - 1) / WPB), 32 * WPB, smem, s>>>(g, T, ph, bs, Ce, factors, status);
  WR_LAUNCH_CHECK();
}

// CTAs of `kern` resident on the whole GPU at `smem` bytes of dynamic shared memory
// (also raises the kernel's dynamic shared memory limit to `smem`).
template <typename Kern>
int persistent_grid(Kern kern, int nth, size_t smem) {
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  WR_CUDA(cudaGetDevice(&dev));
  WR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  WR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nth, smem));
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <int K, int Q, typename FT, int NPGX = 2 * K - 1, int V = 0>
void run_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs, const FT* factors, const double* r,
               double* out, int* err, const double* prev, cudaStream_t s, const ChunkPlan* cp = nullptr) {
  using C = ApplyCfg<K, Q, FT, NPGX, V>;
  const size_t smem = (size_t)C::NS * C::SLOT_ELEMS * sizeof(FT) + sizeof(ApplySmem<K, Q, FT, NPGX, V>);
  auto kern = block_apply_kernel<K, Q, FT, NPGX, V>;
  // persistent grid: CTAs resident on the whole GPU (computed once; thread-safe static)
  static const int grid_cap = persistent_grid(kern, C::NTH, smem);
  const int nblk = bs.kind == 0 ? g.npatch() : 1;
  SingleItems<FT> items{g, bs, factors, r, out, prev};
  items.nblk = nblk;
  items.prev_mode = prev ? 2 : 0;
  int64_t nitems = nblk;
  if (cp && cp->nchunk > 1) {
    items.nchunk = cp->nchunk;
    items.Lc = cp->Lc;
    items.c_first = cp->c_first;
    items.prev_mode = cp->prev_mode;
    items.prev = cp->prev;
    nitems = (int64_t)nblk * (cp->nchunk - cp->c_first);
  }
  const int grid = nitems < grid_cap ? (int)nitems : grid_cap;
  if (nitems <= 0) return;
  kern<<<grid, C::NTH, smem, s>>>(g, T, items, nitems, err);
  WR_LAUNCH_CHECK();
}

template <int K, int Q, typename FT, int NPGX = 2 * K - 1, int V = 0>
void run_bt_apply(const BatchSeg* segs, int nseg, int64_t items, const FeTables& T, const double* r, double* yp,
                  bool coarse, int* err, cudaStream_t s) {
  using C = ApplyCfg<K, Q, FT, NPGX, V>;
  const size_t smem = (size_t)C::NS * C::SLOT_ELEMS * sizeof(FT) + sizeof(ApplySmem<K, Q, FT, NPGX, V>);
  auto kern = bt_block_apply_kernel<K, Q, FT, NPGX, V>;
  static const int grid_cap = persistent_grid(kern, C::NTH, smem);
  if (items <= 0) return;
  const int grid = items < grid_cap ? (int)items : grid_cap;
  kern<<<grid, C::NTH, smem, s>>>(segs, nseg, items, T, r, yp, coarse ? 1 : 0, err);
  WR_LAUNCH_CHECK();
}


template <int K, int Q, typename FT>
void run_warp_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs, const FT* factors, const double* r,
                    double* out, const double* prev, cudaStream_t s, const ChunkPlan* cp) {
  auto kern = warp_apply_kernel<K, Q, FT>;
  const size_t smem = sizeof(WarpSmem<K, Q, FT>) * kWarpTileWarps;
  static const int grid_cap = persistent_grid(kern, 32 * kWarpTileWarps, smem);
  const int nblk = g.npatch();
  SingleItems<FT> items{g, bs, factors, r, out, prev};
  items.nblk = nblk;
  items.prev_mode = prev ? 2 : 0;
  int64_t nitems = nblk;
  if (cp && cp->nchunk > 1) {
    items.nchunk = cp->nchunk;
    items.Lc = cp->Lc;
    items.c_first = cp->c_first;
    items.prev_mode = cp->prev_mode;
    items.prev = cp->prev;
    nitems = (int64_t)nblk * (cp->nchunk - cp->c_first);
  }
  if (nitems <= 0) return;
  const int64_t want = (nitems + kWarpTileWarps - 1) / kWarpTileWarps;
  const int grid = want < grid_cap ? (int)want : grid_cap;
  kern<<<grid, 32 * kWarpTileWarps, smem, s>>>(T, items, nitems);
  WR_LAUNCH_CHECK();
}

template <int K, int Q, typename FT>
void run_bt_warp_apply(const BatchSeg* segs, int nseg, int64_t items, const FeTables& T, const double* r, double* yp,
                       cudaStream_t s) {
  auto kern = bt_warp_apply_kernel<K, Q, FT>;
  const size_t smem = sizeof(WarpSmem<K, Q, FT>) * kWarpTileWarps;
  static const int grid_cap = persistent_grid(kern, 32 * kWarpTileWarps, smem);
  if (items <= 0) return;
  const int64_t want = (items + kWarpTileWarps - 1) / kWarpTileWarps;
  const int grid = want < grid_cap ? (int)want : grid_cap;
  kern<<<grid, 32 * kWarpTileWarps, smem, s>>>(segs, nseg, items, T, r, yp);
  WR_LAUNCH_CHECK();
}

template <typename FT>
void run_warp_bulk_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs, const FT* factors, const double* r,
                         double* out, int* err, const double* prev, cudaStream_t s, const ChunkPlan* cp) {
  auto kern = warp_bulk_apply_kernel<FT>;
  const size_t smem = sizeof(WarpBulkSmem<FT>) * kWarpBulkWarps;
  static const int grid_cap = persistent_grid(kern, 32 * kWarpBulkWarps, smem);
  const int nblk = g.npatch();
  SingleItems<FT> items{g, bs, factors, r, out, prev};
  items.nblk = nblk;
  items.prev_mode = prev ? 2 : 0;
  int64_t nitems = nblk;
  if (cp && cp->nchunk > 1) {
    items.nchunk = cp->nchunk;
    items.Lc = cp->Lc;
    items.c_first = cp->c_first;
    items.prev_mode = cp->prev_mode;
    items.prev = cp->prev;
    nitems = (int64_t)nblk * (cp->nchunk - cp->c_first);
  }
  if (nitems <= 0) return;
  const int64_t want = (nitems + kWarpBulkWarps - 1) / kWarpBulkWarps;
  const int grid = want < grid_cap ? (int)want : grid_cap;
  kern<<<grid, 32 * kWarpBulkWarps, smem, s>>>(T, items, nitems, err);
  WR_LAUNCH_CHECK();
}

template <typename FT>
void run_bt_warp_bulk_apply(const BatchSeg* segs, int nseg, int64_t items, const FeTables& T, const double* r,
                            double* yp, int* err, cudaStream_t s) {
  auto kern = bt_warp_bulk_apply_kernel<FT>;
  const size_t smem = sizeof(WarpBulkSmem<FT>) * kWarpBulkWarps;
  static const int grid_cap = persistent_grid(kern, 32 * kWarpBulkWarps, smem);
  if (items <= 0) return;
  const int64_t want = (items + kWarpBulkWarps - 1) / kWarpBulkWarps;
  const int grid = want < grid_cap ? (int)want : grid_cap;
  kern<<<grid, 32 * kWarpBulkWarps, smem, s>>>(segs, nseg, items, T, r, yp, err);
  WR_LAUNCH_CHECK();
}

template <int K, int Q, typename FT>
void apply_variant(int variant, const LevelGeom& g, const FeTables& T, const BlockSet& bs, const FT* factors,
                   const double* r, double* out, int* err, const double* prev, cudaStream_t s,
                   const ChunkPlan* cp) {
  if (variant < 0) variant = default_apply_variant(K);
  // FP64 DG(1) patch blocks store A10 by segments, which only the CTA tiles read: the warp
  // tiles run as tile 2 there
  if constexpr (ApplyCfg<K, Q, FT>::SPA)
    if (variant == 3 || variant == 4) variant = 2;
  if (variant == 4) {  // the bulk-copy warp tile exists for Q2/Q1 DG(0); elsewhere it is tile 3
    if constexpr (K == 1 && Q == 0) run_warp_bulk_apply<FT>(g, T, bs, factors, r, out, err, prev, s, cp);
    else run_warp_apply<K, Q, FT>(g, T, bs, factors, r, out, prev, s, cp);
  } else if (variant == 3) run_warp_apply<K, Q, FT>(g, T, bs, factors, r, out, prev, s, cp);
  else if (variant == 0) run_apply<K, Q, FT, 2 * K - 1, 0>(g, T, bs, factors, r, out, err, prev, s, cp);
  else if (variant == 1) run_apply<K, Q, FT, 2 * K - 1, 1>(g, T, bs, factors, r, out, err, prev, s, cp);
  else run_apply<K, Q, FT, 2 * K - 1, 2>(g, T, bs, factors, r, out, err, prev, s, cp);
}

template <int K, int Q, typename FT>
void bt_apply_variant(int variant, const BatchSeg* segs, int nseg, int64_t items, const FeTables& T,
                      const double* r, double* yp, int* err, cudaStream_t s) {
  if (variant < 0) variant = default_apply_variant(K);
  if constexpr (ApplyCfg<K, Q, FT>::SPA)  // A10 by segments: CTA tiles only (as apply_variant)
    if (variant == 3 || variant == 4) variant = 2;
  if (variant == 4) {
    if constexpr (K == 1 && Q == 0) run_bt_warp_bulk_apply<FT>(segs, nseg, items, T, r, yp, err, s);
    else run_bt_warp_apply<K, Q, FT>(segs, nseg, items, T, r, yp, s);
  } else if (variant == 3) run_bt_warp_apply<K, Q, FT>(segs, nseg, items, T, r, yp, s);
  else if (variant == 0) run_bt_apply<K, Q, FT, 2 * K - 1, 0>(segs, nseg, items, T, r, yp, false, err, s);
  else if (variant == 1) run_bt_apply<K, Q, FT, 2 * K - 1, 1>(segs, nseg, items, T, r, yp, false, err, s);
  else run_bt_apply<K, Q, FT, 2 * K - 1, 2>(segs, nseg, items, T, r, yp, false, err, s);
}

}  // namespace

void launch_block_factor(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const BlockSet& bs,
                         const void* Ce, void* factors, int precision, int* st, cudaStream_t s, bool check) {
  if (check) WR_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
  const double* Cd = static_cast<const double*>(Ce);
  const float* Cf = static_cast<const float*>(Ce);
#define WR_F(K_, Q_)                                                                                     \
  if (g.k == K_ && g.q == Q_) {                                                                          \
    if (precision == WR_FP32)                                                                            \
      run_factor<K_, Q_, float, float>(g, T, ph, bs, Cf, static_cast<float*>(factors), st, s);           \
    else if (precision == WR_BF16)                                                                       \
      run_factor<K_, Q_, float, __nv_bfloat16>(g, T, ph, bs, Cf, static_cast<__nv_bfloat16*>(factors), st, s); \
    else                                                                                                 \
      run_factor<K_, Q_, double, double>(g, T, ph, bs, Cd, static_cast<double*>(factors), st, s);        \
  } else
  if (bs.kind == 1 && g.k == 1 && bs.npg == 4) {  // coarse 3x3 block of Q2/Q1 (FP64)
    if (g.q == 0) run_factor<1, 0, double, double, 4>(g, T, ph, bs, Cd, static_cast<double*>(factors), st, s);
    else run_factor<1, 1, double, double, 4>(g, T, ph, bs, Cd, static_cast<double*>(factors), st, s);
  } else if (bs.kind == 0 && g.k == 1 && g.q == 0 && precision == WR_FP32) {  // a warp per block
    run_factor_warp<float>(g, T, ph, bs, Cf, static_cast<float*>(factors), st, s);
  } else if (bs.kind == 0 && g.k == 1 && g.q == 0 && precision == WR_BF16) {
    run_factor_warp<__nv_bfloat16>(g, T, ph, bs, Cf, static_cast<__nv_bfloat16*>(factors), st, s);
  } else
  if (g.q == 2 || g.q == 3) {  // DG(2), DG(3): FP64
    if (precision != WR_FP64) throw WrError(WR_ERR_ARG, "DG(2) and DG(3) factors are FP64 only");
    double* f = static_cast<double*>(factors);
    if (g.k == 1 && g.q == 2) run_factor<1, 2, double, double>(g, T, ph, bs, Cd, f, st, s);
    else if (g.k == 1) run_factor<1, 3, double, double>(g, T, ph, bs, Cd, f, st, s);
    else if (g.q == 2) run_factor<2, 2, double, double>(g, T, ph, bs, Cd, f, st, s);
    else run_factor<2, 3, double, double>(g, T, ph, bs, Cd, f, st, s);
  } else
  WR_F(1, 0) WR_F(1, 1) WR_F(2, 0) WR_F(2, 1) throw WrError(WR_ERR_ARG, "unsupported (k, q)");
#undef WR_F
  if (!check) return;
  int h = 0;
  WR_CUDA(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  WR_CUDA(cudaStreamSynchronize(s));
  if (h) throw WrError(WR_ERR_NAN, "singular patch block (zero pivot) in the factorisation");
}

void launch_block_apply(const LevelGeom& g, const FeTables& T, const BlockSet& bs, const void* factors, int precision,
                        const double* r, double* out, int* err, cudaStream_t s, const double* prev, int variant,
                        const ChunkPlan* cp) {
#define WR_A(K_, Q_)                                                                                   \
  if (g.k == K_ && g.q == Q_) {                                                                        \
    if (bs.kind == 1) {                                                                                \
      run_apply<K_, Q_, double>(g, T, bs, static_cast<const double*>(factors), r, out, err, prev, s);  \
    } else if (precision == WR_FP32) {                                                                 \
      apply_variant<K_, Q_, float>(variant, g, T, bs, static_cast<const float*>(factors), r, out, err, prev, s, cp); \
    } else if (precision == WR_BF16) {                                                                 \
      apply_variant<K_, Q_, __nv_bfloat16>(variant, g, T, bs, static_cast<const __nv_bfloat16*>(factors), r, out, \
                                           err, prev, s, cp);                                          \
    } else {                                                                                           \
      apply_variant<K_, Q_, double>(variant, g, T, bs, static_cast<const double*>(factors), r, out, err, prev, s, cp); \
    }                                                                                                  \
  } else
  if (bs.kind == 1 && g.k == 1 && bs.npg == 4) {  // coarse 3x3 block of Q2/Q1 (FP64)
    if (g.q == 0) run_apply<1, 0, double, 4>(g, T, bs, static_cast<const double*>(factors), r, out, err, prev, s);
    else run_apply<1, 1, double, 4>(g, T, bs, static_cast<const double*>(factors), r, out, err, prev, s);
  } else
  if (g.q == 2 || g.q == 3) {  // DG(2), DG(3): FP64, CTA tile 0
    if (precision != WR_FP64) throw WrError(WR_ERR_ARG, "DG(2) and DG(3) factors are FP64 only");
    const double* f = static_cast<const double*>(factors);
    const ChunkPlan* c2 = bs.kind == 0 ? cp : nullptr;
    if (g.k == 1 && g.q == 2) run_apply<1, 2, double>(g, T, bs, f, r, out, err, prev, s, c2);
    else if (g.k == 1) run_apply<1, 3, double>(g, T, bs, f, r, out, err, prev, s, c2);
    else if (g.q == 2) run_apply<2, 2, double>(g, T, bs, f, r, out, err, prev, s, c2);
    else run_apply<2, 3, double>(g, T, bs, f, r, out, err, prev, s, c2);
  } else
  WR_A(1, 0) WR_A(1, 1) WR_A(2, 0) WR_A(2, 1) throw WrError(WR_ERR_ARG, "unsupported (k, q)");
#undef WR_A
}

void launch_scatter(const LevelGeom& g, const BlockSet& bs, const double* Yp, double* y, cudaStream_t s) {
  const int threads = 256, wt = bs.weighted;
  const unsigned blocks = (unsigned)((g.ndofs + threads - 1) / threads);
  if (g.k == 1 && g.q == 0) scatter_kernel<1, 0><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 1 && g.q == 1) scatter_kernel<1, 1><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 2 && g.q == 0) scatter_kernel<2, 0><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 2 && g.q == 1) scatter_kernel<2, 1><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 1 && g.q == 2) scatter_kernel<1, 2><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 1 && g.q == 3) scatter_kernel<1, 3><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 2 && g.q == 2) scatter_kernel<2, 2><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else if (g.k == 2 && g.q == 3) scatter_kernel<2, 3><<<blocks, threads, 0, s>>>(g, Yp, y, wt);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
  WR_LAUNCH_CHECK();
}

namespace {
__global__ void patch_slots_kernel(LevelGeom g, BlockSet bs, int blk, int* __restrict__ out) {
  for (int s = threadIdx.x; s < bs.ms; s += blockDim.x) out[s] = decode_slot(g, bs, blk, s).sp;
}
}  // namespace

// Spatial index of every slot of block `blk` as the kernels decode it (-1 = padding).
void launch_patch_slots(const LevelGeom& g, const BlockSet& bs, int blk, int* out_sp, cudaStream_t s) {
  patch_slots_kernel<<<1, 128, 0, s>>>(g, bs, blk, out_sp);
  WR_LAUNCH_CHECK();
}

void bt_block_apply(int k, int q, int precision, const BatchSeg* segs, int nseg, int64_t items, int64_t dofs,
                    const FeTables& T, const double* r, double* out, double* yp, int* err, int coarse_n,
                    cudaStream_t s, int variant) {
  // coarse blocks (coarse_n = 2 or 3) are FP64; the 3x3 coarse block of Q2/Q1 uses its own slot shape
  if (coarse_n == 3) {
    if (k != 1) throw WrError(WR_ERR_ARG, "3x3 coarse blocks need k = 1");
    if (q == 0) run_bt_apply<1, 0, double, 4>(segs, nseg, items, T, r, yp, true, err, s);
    else run_bt_apply<1, 1, double, 4>(segs, nseg, items, T, r, yp, true, err, s);
    return;
  }
  if (coarse_n == 2) {
    if (k == 1 && q == 0) run_bt_apply<1, 0, double>(segs, nseg, items, T, r, yp, true, err, s);
    else if (k == 1 && q == 1) run_bt_apply<1, 1, double>(segs, nseg, items, T, r, yp, true, err, s);
    else if (k == 2 && q == 0) run_bt_apply<2, 0, double>(segs, nseg, items, T, r, yp, true, err, s);
    else if (k == 2 && q == 1) run_bt_apply<2, 1, double>(segs, nseg, items, T, r, yp, true, err, s);
    else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
    return;
  }
#define WR_BA(K_, Q_)                                                                                    \
  if (k == K_ && q == Q_) {                                                                              \
    if (precision == WR_FP32) bt_apply_variant<K_, Q_, float>(variant, segs, nseg, items, T, r, yp, err, s); \
    else if (precision == WR_BF16)                                                                       \
      bt_apply_variant<K_, Q_, __nv_bfloat16>(variant, segs, nseg, items, T, r, yp, err, s);             \
    else bt_apply_variant<K_, Q_, double>(variant, segs, nseg, items, T, r, yp, err, s);                 \
  } else
  WR_BA(1, 0) WR_BA(1, 1) WR_BA(2, 0) WR_BA(2, 1) throw WrError(WR_ERR_ARG, "unsupported (k, q)");
#undef WR_BA
  if (dofs <= 0) return;
  const unsigned blocks = (unsigned)((dofs + 255) / 256);
  if (k == 1 && q == 0) bt_scatter_kernel<1, 0><<<blocks, 256, 0, s>>>(segs, nseg, dofs, yp, out);
  else if (k == 1 && q == 1) bt_scatter_kernel<1, 1><<<blocks, 256, 0, s>>>(segs, nseg, dofs, yp, out);
  else if (k == 2 && q == 0) bt_scatter_kernel<2, 0><<<blocks, 256, 0, s>>>(segs, nseg, dofs, yp, out);
  else bt_scatter_kernel<2, 1><<<blocks, 256, 0, s>>>(segs, nseg, dofs, yp, out);
  WR_LAUNCH_CHECK();
}


// ---------------------------------------------------------------- self-test of the bounded wait
// One thread initialises an mbarrier that nothing ever completes and waits on it
// with the apply kernels' bounded wait; it must give up and report it.
__global__ void bounded_wait_selftest_kernel(int* timed_out, unsigned long long* ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const unsigned long long t0 = global_ns();
  const bool ok = mbar_wait_bounded(smem_u32(&bar), 0);
  *ns = global_ns() - t0;
  *timed_out = ok ? 0 : 1;
}

void launch_bounded_wait_selftest(int* timed_out, unsigned long long* ns, cudaStream_t s) {
  bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(timed_out, ns);
  WR_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- time-parallel patch solve
// The partitioned forward substitution of Sec. 5's cost model: each patch's slabs are
// split into chunks; (A) every chunk is swept from a zero jump state, all chunks at
// once; (B) the chunk-end states are chained through the chunks' transfer matrices
// T_c (the chunk's response to a unit incoming velocity state, built at setup by
// sweeps from unit states): carry_c = e_c + T_c carry_{c-1}; (C) every chunk but the
// first is swept again from its incoming state.

__global__ void cr_unit_kernel(int64_t n, int nt, int ms, int j, double* __restrict__ buf) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int s = int(idx % ms), a = int((idx / ms) % nt);
  buf[idx] = (a == nt - 1 && s == j) ? 1.0 : 0.0;
}

__global__ void cr_gather_kernel(int npatch, int nchunk, int Lc, int N, int nt, int ms, int mv, int j,
                                 const double* __restrict__ Yp, double* __restrict__ Tm) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npatch * nchunk * mv) return;
  const int i = int(idx % mv);
  const int64_t bc = idx / mv;
  const int c = int(bc % nchunk), blk = int(bc / nchunk);
  const int e = min((c + 1) * Lc, N) - 1;
  Tm[(((int64_t)blk * nchunk + c) * mv + i) * mv + j] = Yp[(((int64_t)e * npatch + blk) * nt + nt - 1) * ms + i];
}

// one CTA per patch, one thread per velocity slot of the state
__global__ void cr_carry_kernel(int npatch, int nchunk, int Lc, int N, int nt, int ms, int mv,
                                const double* __restrict__ Tm, const double* __restrict__ Yp,
                                double* __restrict__ carry) {
  extern __shared__ double st[];  // mv doubles
  const int blk = blockIdx.x, i = threadIdx.x;
  if (i < mv) st[i] = 0.0;
  __syncthreads();
  const int64_t slab_out = (int64_t)npatch * nt * ms;
  for (int c = 0; c + 1 < nchunk; ++c) {
    const int e = min((c + 1) * Lc, N) - 1;
    double v = 0.0;
    if (i < mv) {
      v = Yp[(((int64_t)e * npatch + blk) * nt + nt - 1) * ms + i];
      const double* T = Tm + ((int64_t)blk * nchunk + c) * mv * mv + (int64_t)i * mv;
      for (int jj = 0; jj < mv; ++jj) v = fma(T[jj], st[jj], v);
    }
    __syncthreads();
    if (i < mv) {
      st[i] = v;
      carry[c * slab_out + ((int64_t)blk * nt + nt - 1) * ms + i] = v;
    }
    __syncthreads();
  }
}

void cr_unit_state(const LevelGeom& g, const BlockSet& bs, int j, double* buf, cudaStream_t s) {
  const int64_t n = (int64_t)g.npatch() * g.nt * bs.ms;
  cr_unit_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, g.nt, bs.ms, j, buf);
  WR_LAUNCH_CHECK();
}

void cr_gather_column(const LevelGeom& g, const BlockSet& bs, int nchunk, int Lc, int j, const double* Yp,
                      double* Tm, cudaStream_t s) {
  const int mv = 2 * bs.nvg * bs.nvg;
  const int64_t n = (int64_t)g.npatch() * nchunk * mv;
  cr_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.npatch(), nchunk, Lc, g.N, g.nt, bs.ms, mv, j, Yp,
                                                               Tm);
  WR_LAUNCH_CHECK();
}

void cr_carry(const LevelGeom& g, const BlockSet& bs, int nchunk, int Lc, const double* Tm, const double* Yp,
              double* carry, cudaStream_t s) {
  const int mv = 2 * bs.nvg * bs.nvg;
  const int nth = (mv + 31) / 32 * 32;
  cr_carry_kernel<<<g.npatch(), nth, sizeof(double) * mv, s>>>(g.npatch(), nchunk, Lc, g.N, g.nt, bs.ms, mv, Tm, Yp,
                                                                carry);
  WR_LAUNCH_CHECK();
}
