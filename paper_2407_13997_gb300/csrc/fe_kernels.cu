// Space-time residual F(U) and Jacobian action J(W) x of Eq. nsfem, sum-factorised
// and matrix-free on the uniform quadrilateral mesh (hot-path step (e)), plus the
// element convection matrices used by the patch assembly, boundary data and the
// injection of the linearisation point to coarser levels.
//
// Element kernel: one warp per (cell, slab).  The warp stages the element's
// nodal data in shared memory, interpolates every field to the (k+3)^2 Gauss
// points by two 1D passes (x, then y), forms the pointwise coefficients of the
// weak form, and contracts them against the test functions by the transposed
// two passes.  Element results go to a per-element buffer that a second kernel
// sums into the global vector in a fixed order (deterministic, no atomics).
//
// Per slab n and test psi = tau_a phi (velocity component c), chi (pressure):
//   value coefficient  sum_b Kt[a,b] u_{c,b} - tau_a(0) u^-_c
//                      + dt conv sum_{b,e} T3[a,b,e] (convection term)
//                      - dt sum_g wt_g tau_a(t_g) f_c(t_g)               (F only)
//   gradient coeff.    dt sum_b Wt[a,b] (nu grad u_{c,b} + Phi_b e_c)
//   pressure coeff.    dt sum_b Wt[a,b] div u_b
// with the convection term (U_b.grad) U_{c,e} for F and
// (W_b.grad) x_{c,e} + (x_b.grad) W_{c,e} for J.
#include <cmath>
#include <mutex>

#include "wrmg_internal.h"

namespace {

template <int K, int Q>
struct D {
  static constexpr int NT = Q + 1, NVL = K + 2, NPL = K + 1, NQ = K + 3;
  static constexpr int NVE = NVL * NVL, NPE = NPL * NPL, NQ2 = NQ * NQ;
  static constexpr int ELEM = NT * (2 * NVE + NPE);
};

constexpr int kWarps = 4;  // elements per CTA

__device__ __forceinline__ void exact_velocity(const PhysParams& ph, double x, double y, double t,
                                               double& ux, double& uy) {
  if (ph.kind == WR_TAYLOR_GREEN) {
    const double e = exp(-2.0 * ph.nu * M_PI * M_PI * t);
    ux = -cospi(x) * sinpi(y) * e;
    uy = sinpi(x) * cospi(y) * e;
  } else if (ph.kind == WR_POLY) {
    const double s = ph.steady ? 1.0 : 1.0 + t;
    ux = y * y * s;
    uy = x * x * s;
  } else {
    ux = 0.0;
    uy = 0.0;
  }
}

// Dirichlet data at velocity node (gx, gy) of a level with nv nodes per direction:
// the exact solution, except for the lid-driven cavity (u = (1, 0) on the open top
// edge, zero on the other walls and at the top corners).
__device__ __forceinline__ void dirichlet_velocity(const PhysParams& ph, int gx, int gy, int nv, double hn, double t,
                                                   double& ux, double& uy) {
  if (ph.kind == WR_LID) {
    ux = (gy == nv - 1 && gx > 0 && gx < nv - 1) ? 1.0 : 0.0;
    uy = 0.0;
  } else {
    exact_velocity(ph, gx * hn, gy * hn, t, ux, uy);
  }
}

__device__ __forceinline__ void forcing(const PhysParams& ph, double x, double y, double t, double& fx,
                                        double& fy) {
  if (ph.kind == WR_POLY) {
    const double nu = ph.nu, c = ph.conv;
    if (ph.steady) {
      fx = 2.0 * c * x * x * y + 1.0 - 2.0 * nu;
      fy = 2.0 * c * x * y * y + 1.0 - 2.0 * nu;
    } else {
      const double s = 1.0 + t;
      fx = y * y + 2.0 * c * x * x * y * s * s + 1.0 - 2.0 * nu * s;
      fy = x * x + 2.0 * c * x * y * y * s * s + 1.0 - 2.0 * nu * s;
    }
  } else if (ph.kind == WR_FOURIER) {
    fx = 0.0;
    fy = 0.0;
    for (int m = 0; m < ph.n_modes; ++m) {
      const double a = ph.amp[m] * M_PI;
      const double sx = sinpi(ph.mx[m] * x), cx = cospi(ph.mx[m] * x);
      const double sy = sinpi(ph.my[m] * y), cy = cospi(ph.my[m] * y);
      fx += a * ph.my[m] * sx * cy;
      fy -= a * ph.mx[m] * cx * sy;
    }
  } else {
    fx = 0.0;
    fy = 0.0;
  }
}

__device__ __forceinline__ bool vel_dirichlet(const LevelGeom& g, int gx, int gy) {
  return gx == 0 || gy == 0 || gx == g.nv - 1 || gy == g.nv - 1;
}

// Shared-memory workspace of one element (one warp).
template <int K, int Q, bool LIN>
struct ElemSmem {
  using d = D<K, Q>;
  // velocity fields: u(c,b) [2 NT], w(c,b) [2 NT, J only], u^-(c) [2]
  static constexpr int FV = LIN ? 4 * d::NT + 2 : 2 * d::NT + 2;
  static constexpr int FU = 0, FW = 2 * d::NT, FUP = LIN ? 4 * d::NT : 2 * d::NT;
  double vn[FV][d::NVE];           // nodal velocity fields
  double pn[d::NT][d::NPE];        // nodal pressure
  double t1[FV][2][d::NVL][d::NQ]; // x-pass values / derivatives
  double vq[FV][3][d::NQ2];        // value, d/dx, d/dy at Gauss points
  double pq[d::NT][d::NQ2];
  double cv[2 * d::NT][3][d::NQ2]; // output coefficients (value, x-grad, y-grad)
  double cp[d::NT][d::NQ2];
  double out[d::ELEM];
};

// One warp computes the element contribution of (cell, slab) for F (LIN = false)
// or J x (LIN = true).  `x` is U for F.
template <int K, int Q, bool LIN>
__device__ __forceinline__ void element_body(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                                             const double* __restrict__ W, const double* __restrict__ x,
                                             double* __restrict__ ye, int cell, int slab) {
  using d = D<K, Q>;
  using SM = ElemSmem<K, Q, LIN>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM& s = reinterpret_cast<SM*>(smem_raw)[threadIdx.x / 32];
  const int lane = threadIdx.x & 31;
  const int CI = cell % g.n, CJ = cell / g.n;
  const double h = g.h, dt = g.dt;
  const int nv = g.nv, np = g.np, S = g.S;
  const int64_t nv2 = (int64_t)nv * nv;

  // ---- gather nodal data
  for (int it = lane; it < 2 * d::NVE; it += 32) {
    const int c = it / d::NVE, l = it % d::NVE;
    const int gx = CI * (K + 1) + l % d::NVL, gy = CJ * (K + 1) + l / d::NVL;
    const int64_t sp = c * nv2 + (int64_t)gy * nv + gx;
    const bool dir = vel_dirichlet(g, gx, gy);
    for (int b = 0; b < d::NT; ++b) {
      const int64_t off = ((int64_t)slab * d::NT + b) * S + sp;
      s.vn[SM::FU + c * d::NT + b][l] = (LIN && dir) ? 0.0 : x[off];
      if constexpr (LIN) s.vn[SM::FW + c * d::NT + b][l] = W[off];
    }
    double up;
    if (slab > 0) {
      const int64_t off = ((int64_t)(slab - 1) * d::NT + (d::NT - 1)) * S + sp;
      up = (LIN && dir) ? 0.0 : x[off];
    } else if (LIN) {
      up = 0.0;
    } else if (ph.u0) {
      up = ph.u0[sp];
    } else {
      double ux, uy;
      exact_velocity(ph, gx * (h / (K + 1)), gy * (h / (K + 1)), ph.t0, ux, uy);
      up = c == 0 ? ux : uy;
    }
    s.vn[SM::FUP + c][l] = up;
  }
  for (int it = lane; it < d::NT * d::NPE; it += 32) {
    const int b = it / d::NPE, l = it % d::NPE;
    const int px = CI * K + l % d::NPL, py = CJ * K + l / d::NPL;
    s.pn[b][l] = x[((int64_t)slab * d::NT + b) * S + 2 * nv2 + (int64_t)py * np + px];
  }
  __syncwarp();

  // ---- interpolation to Gauss points: x pass
  for (int it = lane; it < SM::FV * d::NVL * d::NQ; it += 32) {
    const int f = it / (d::NVL * d::NQ), r = it % (d::NVL * d::NQ);
    const int j = r / d::NQ, qx = r % d::NQ;
    double v = 0.0, dv = 0.0;
#pragma unroll
    for (int i = 0; i < d::NVL; ++i) {
      const double u = s.vn[f][j * d::NVL + i];
      v = fma(T.Bv[qx][i], u, v);
      dv = fma(T.Dv[qx][i], u, dv);
    }
    s.t1[f][0][j][qx] = v;
    s.t1[f][1][j][qx] = dv;
  }
  for (int it = lane; it < d::NT * d::NQ2; it += 32) {  // pressure values, direct 2D sum
    const int b = it / d::NQ2, q = it % d::NQ2;
    const int qy = q / d::NQ, qx = q % d::NQ;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < d::NPL; ++j)
#pragma unroll
      for (int i = 0; i < d::NPL; ++i) v = fma(T.Bp[qy][j] * T.Bp[qx][i], s.pn[b][j * d::NPL + i], v);
    s.pq[b][q] = v;
  }
  __syncwarp();
  // y pass
  const double ih = 1.0 / h;
  for (int it = lane; it < SM::FV * d::NQ2; it += 32) {
    const int f = it / d::NQ2, q = it % d::NQ2;
    const int qy = q / d::NQ, qx = q % d::NQ;
    double v = 0.0, vx = 0.0, vy = 0.0;
#pragma unroll
    for (int j = 0; j < d::NVL; ++j) {
      v = fma(T.Bv[qy][j], s.t1[f][0][j][qx], v);
      vx = fma(T.Bv[qy][j], s.t1[f][1][j][qx], vx);
      vy = fma(T.Dv[qy][j], s.t1[f][0][j][qx], vy);
    }
    s.vq[f][0][q] = v;
    s.vq[f][1][q] = vx * ih;
    s.vq[f][2][q] = vy * ih;
  }
  __syncwarp();

  // ---- pointwise coefficients
  for (int q = lane; q < d::NQ2; q += 32) {
    const int qy = q / d::NQ, qx = q % d::NQ;
    const double om = T.wq[qx] * T.wq[qy] * h * h;
    double fxg[WR_MAX_NTQ], fyg[WR_MAX_NTQ];
    if constexpr (!LIN) {
      const double xx = (CI + T.xq[qx]) * h, yy = (CJ + T.xq[qy]) * h;
      for (int gq = 0; gq < Q + 2; ++gq)
        forcing(ph, xx, yy, ph.t0 + (slab + T.tq[gq]) * dt, fxg[gq], fyg[gq]);
    }
#pragma unroll
    for (int a = 0; a < d::NT; ++a) {
      double pw = 0.0, divw = 0.0;
#pragma unroll
      for (int b = 0; b < d::NT; ++b) {
        pw = fma(T.Wt[a][b], s.pq[b][q], pw);
        divw = fma(T.Wt[a][b], s.vq[SM::FU + 0 * d::NT + b][1][q] + s.vq[SM::FU + 1 * d::NT + b][2][q], divw);
      }
      s.cp[a][q] = om * dt * divw;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        double val = -T.tau0[a] * s.vq[SM::FUP + c][0][q];
        double gx = 0.0, gy = 0.0, cv = 0.0;
#pragma unroll
        for (int b = 0; b < d::NT; ++b) {
          const int fu = SM::FU + c * d::NT + b;
          val = fma(T.Kt[a][b], s.vq[fu][0][q], val);
          gx = fma(T.Wt[a][b], s.vq[fu][1][q], gx);
          gy = fma(T.Wt[a][b], s.vq[fu][2][q], gy);
#pragma unroll
          for (int e = 0; e < d::NT; ++e) {
            const double t3 = T.T3[a][b][e];
            const int fe = SM::FU + c * d::NT + e;
            if constexpr (LIN) {
              const int wb = SM::FW + b, wb1 = SM::FW + d::NT + b;     // W_b components
              const int ub = SM::FU + b, ub1 = SM::FU + d::NT + b;     // x_b components
              const int we = SM::FW + c * d::NT + e;
              const double term = s.vq[wb][0][q] * s.vq[fe][1][q] + s.vq[wb1][0][q] * s.vq[fe][2][q] +
                                  s.vq[ub][0][q] * s.vq[we][1][q] + s.vq[ub1][0][q] * s.vq[we][2][q];
              cv = fma(t3, term, cv);
            } else {
              const int ub = SM::FU + b, ub1 = SM::FU + d::NT + b;
              const double term = s.vq[ub][0][q] * s.vq[fe][1][q] + s.vq[ub1][0][q] * s.vq[fe][2][q];
              cv = fma(t3, term, cv);
            }
          }
        }
        val = fma(dt * ph.conv, cv, val);
        if constexpr (!LIN) {
          double fsum = 0.0;
          for (int gq = 0; gq < Q + 2; ++gq) fsum += T.wtq[gq] * T.Tq[a][gq] * (c == 0 ? fxg[gq] : fyg[gq]);
          val -= dt * fsum;
        }
        gx = dt * ph.nu * gx + (c == 0 ? dt * pw : 0.0);
        gy = dt * ph.nu * gy + (c == 1 ? dt * pw : 0.0);
        s.cv[c * d::NT + a][0][q] = om * val;
        s.cv[c * d::NT + a][1][q] = om * gx * ih;
        s.cv[c * d::NT + a][2][q] = om * gy * ih;
      }
    }
  }
  __syncwarp();

  // ---- test contraction: y pass (reuse t1 for the 2 NT output fields)
  for (int it = lane; it < 2 * d::NT * d::NVL * d::NQ; it += 32) {
    const int f = it / (d::NVL * d::NQ), r = it % (d::NVL * d::NQ);
    const int j = r / d::NQ, qx = r % d::NQ;
    double a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int qy = 0; qy < d::NQ; ++qy) {
      const int q = qy * d::NQ + qx;
      a1 = fma(T.Bv[qy][j], s.cv[f][0][q], a1);
      a1 = fma(T.Dv[qy][j], s.cv[f][2][q], a1);
      a2 = fma(T.Bv[qy][j], s.cv[f][1][q], a2);
    }
    s.t1[f][0][j][qx] = a1;
    s.t1[f][1][j][qx] = a2;
  }
  __syncwarp();
  // x pass -> element output; layout a*(2 NVE + NPE) + c*NVE + l, then pressure
  for (int it = lane; it < 2 * d::NT * d::NVE; it += 32) {
    const int f = it / d::NVE, l = it % d::NVE;
    const int c = f / d::NT, a = f % d::NT;
    const int j = l / d::NVL, i = l % d::NVL;
    double v = 0.0;
#pragma unroll
    for (int qx = 0; qx < d::NQ; ++qx) {
      v = fma(T.Bv[qx][i], s.t1[f][0][j][qx], v);
      v = fma(T.Dv[qx][i], s.t1[f][1][j][qx], v);
    }
    s.out[a * (2 * d::NVE + d::NPE) + c * d::NVE + l] = v;
  }
  for (int it = lane; it < d::NT * d::NPE; it += 32) {
    const int a = it / d::NPE, l = it % d::NPE;
    const int j = l / d::NPL, i = l % d::NPL;
    double v = 0.0;
    for (int qy = 0; qy < d::NQ; ++qy)
      for (int qx = 0; qx < d::NQ; ++qx)
        v = fma(T.Bp[qy][j] * T.Bp[qx][i], s.cp[a][qy * d::NQ + qx], v);
    s.out[a * (2 * d::NVE + d::NPE) + 2 * d::NVE + l] = v;
  }
  __syncwarp();
  double* dst = ye + ((int64_t)slab * g.ncells() + cell) * d::ELEM;
  for (int it = lane; it < d::ELEM; it += 32) dst[it] = s.out[it];
}

// ---------------------------------------------------------------- FP32 Jacobian action
// J(W) x in single precision for the reduced-precision forms, where it only feeds the
// smoother's residuals inside the V-cycle (the Newton residual and the outer FGMRES
// keep the FP64 kernel above).  Same algorithm as element_body<.., LIN = true>, with
// the reference tables staged once per CTA as floats; element results stay FP64 in
// the per-element buffer, so the assembly is unchanged.
template <int K, int Q>
struct TabF {
  using d = D<K, Q>;
  float Bv[d::NQ][d::NVL], Dv[d::NQ][d::NVL], Bp[d::NQ][d::NPL], wq[d::NQ];
  float Kt[d::NT][d::NT], Wt[d::NT][d::NT], T3[d::NT][d::NT][d::NT], tau0[d::NT];
};

template <int K, int Q>
struct ElemSmemF {
  using d = D<K, Q>;
  static constexpr int FV = 4 * d::NT + 2;
  static constexpr int FU = 0, FW = 2 * d::NT, FUP = 4 * d::NT;
  float vn[FV][d::NVE];
  float pn[d::NT][d::NPE];
  float t1[FV][2][d::NVL][d::NQ];
  float vq[FV][3][d::NQ2];
  float pq[d::NT][d::NQ2];
  float cv[2 * d::NT][3][d::NQ2];
  float cp[d::NT][d::NQ2];
  float out[d::ELEM];
};

template <int K, int Q>
__device__ __forceinline__ void stage_tab_f(const FeTables& T, TabF<K, Q>& tb) {
  using d = D<K, Q>;
  for (int e = threadIdx.x; e < d::NQ * d::NVL; e += blockDim.x) {
    const int q = e / d::NVL, i = e % d::NVL;
    tb.Bv[q][i] = (float)T.Bv[q][i];
    tb.Dv[q][i] = (float)T.Dv[q][i];
  }
  for (int e = threadIdx.x; e < d::NQ * d::NPL; e += blockDim.x) tb.Bp[e / d::NPL][e % d::NPL] = (float)T.Bp[e / d::NPL][e % d::NPL];
  for (int e = threadIdx.x; e < d::NQ; e += blockDim.x) tb.wq[e] = (float)T.wq[e];
  for (int e = threadIdx.x; e < d::NT * d::NT * d::NT; e += blockDim.x) {
    const int a = e / (d::NT * d::NT), b = (e / d::NT) % d::NT, c = e % d::NT;
    tb.T3[a][b][c] = (float)T.T3[a][b][c];
    if (c == 0) {
      tb.Kt[a][b] = (float)T.Kt[a][b];
      tb.Wt[a][b] = (float)T.Wt[a][b];
    }
  }
  for (int e = threadIdx.x; e < d::NT; e += blockDim.x) tb.tau0[e] = (float)T.tau0[e];
}

template <int K, int Q>
__device__ __forceinline__ void element_body_f32(const LevelGeom& g, const TabF<K, Q>& tb, const PhysParams& ph,
                                                 const double* __restrict__ W, const double* __restrict__ x,
                                                 double* __restrict__ ye, ElemSmemF<K, Q>& s, int cell, int slab) {
  using d = D<K, Q>;
  using SM = ElemSmemF<K, Q>;
  const int lane = threadIdx.x & 31;
  const int CI = cell % g.n, CJ = cell / g.n;
  const float h = (float)g.h, dt = (float)g.dt;
  const int nv = g.nv, np = g.np, S = g.S;
  const int64_t nv2 = (int64_t)nv * nv;
  for (int it = lane; it < 2 * d::NVE; it += 32) {
    const int c = it / d::NVE, l = it % d::NVE;
    const int gx = CI * (K + 1) + l % d::NVL, gy = CJ * (K + 1) + l / d::NVL;
    const int64_t sp = c * nv2 + (int64_t)gy * nv + gx;
    const bool dir = vel_dirichlet(g, gx, gy);
    for (int b = 0; b < d::NT; ++b) {
      const int64_t off = ((int64_t)slab * d::NT + b) * S + sp;
      s.vn[SM::FU + c * d::NT + b][l] = dir ? 0.f : (float)x[off];
      s.vn[SM::FW + c * d::NT + b][l] = (float)W[off];
    }
    float up = 0.f;
    if (slab > 0 && !dir) up = (float)x[((int64_t)(slab - 1) * d::NT + (d::NT - 1)) * S + sp];
    s.vn[SM::FUP + c][l] = up;
  }
  for (int it = lane; it < d::NT * d::NPE; it += 32) {
    const int b = it / d::NPE, l = it % d::NPE;
    const int px = CI * K + l % d::NPL, py = CJ * K + l / d::NPL;
    s.pn[b][l] = (float)x[((int64_t)slab * d::NT + b) * S + 2 * nv2 + (int64_t)py * np + px];
  }
  __syncwarp();
  for (int it = lane; it < SM::FV * d::NVL * d::NQ; it += 32) {
    const int f = it / (d::NVL * d::NQ), r = it % (d::NVL * d::NQ);
    const int j = r / d::NQ, qx = r % d::NQ;
    float v = 0.f, dv = 0.f;
#pragma unroll
    for (int i = 0; i < d::NVL; ++i) {
      const float u = s.vn[f][j * d::NVL + i];
      v = fmaf(tb.Bv[qx][i], u, v);
      dv = fmaf(tb.Dv[qx][i], u, dv);
    }
    s.t1[f][0][j][qx] = v;
    s.t1[f][1][j][qx] = dv;
  }
  for (int it = lane; it < d::NT * d::NQ2; it += 32) {
    const int b = it / d::NQ2, q = it % d::NQ2;
    const int qy = q / d::NQ, qx = q % d::NQ;
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < d::NPL; ++j)
#pragma unroll
      for (int i = 0; i < d::NPL; ++i) v = fmaf(tb.Bp[qy][j] * tb.Bp[qx][i], s.pn[b][j * d::NPL + i], v);
    s.pq[b][q] = v;
  }
  __syncwarp();
  const float ih = 1.f / h;
  for (int it = lane; it < SM::FV * d::NQ2; it += 32) {
    const int f = it / d::NQ2, q = it % d::NQ2;
    const int qy = q / d::NQ, qx = q % d::NQ;
    float v = 0.f, vx = 0.f, vy = 0.f;
#pragma unroll
    for (int j = 0; j < d::NVL; ++j) {
      v = fmaf(tb.Bv[qy][j], s.t1[f][0][j][qx], v);
      vx = fmaf(tb.Bv[qy][j], s.t1[f][1][j][qx], vx);
      vy = fmaf(tb.Dv[qy][j], s.t1[f][0][j][qx], vy);
    }
    s.vq[f][0][q] = v;
    s.vq[f][1][q] = vx * ih;
    s.vq[f][2][q] = vy * ih;
  }
  __syncwarp();
  const float nu = (float)ph.nu, conv = (float)ph.conv;
  for (int q = lane; q < d::NQ2; q += 32) {
    const int qy = q / d::NQ, qx = q % d::NQ;
    const float om = tb.wq[qx] * tb.wq[qy] * h * h;
#pragma unroll
    for (int a = 0; a < d::NT; ++a) {
      float pw = 0.f, divw = 0.f;
#pragma unroll
      for (int b = 0; b < d::NT; ++b) {
        pw = fmaf(tb.Wt[a][b], s.pq[b][q], pw);
        divw = fmaf(tb.Wt[a][b], s.vq[SM::FU + 0 * d::NT + b][1][q] + s.vq[SM::FU + 1 * d::NT + b][2][q], divw);
      }
      s.cp[a][q] = om * dt * divw;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float val = -tb.tau0[a] * s.vq[SM::FUP + c][0][q];
        float gx = 0.f, gy = 0.f, cv = 0.f;
#pragma unroll
        for (int b = 0; b < d::NT; ++b) {
          const int fu = SM::FU + c * d::NT + b;
          val = fmaf(tb.Kt[a][b], s.vq[fu][0][q], val);
          gx = fmaf(tb.Wt[a][b], s.vq[fu][1][q], gx);
          gy = fmaf(tb.Wt[a][b], s.vq[fu][2][q], gy);
#pragma unroll
          for (int e = 0; e < d::NT; ++e) {
            const int fe = SM::FU + c * d::NT + e;
            const int wb = SM::FW + b, wb1 = SM::FW + d::NT + b;
            const int ub = SM::FU + b, ub1 = SM::FU + d::NT + b;
            const int we = SM::FW + c * d::NT + e;
            const float term = s.vq[wb][0][q] * s.vq[fe][1][q] + s.vq[wb1][0][q] * s.vq[fe][2][q] +
                               s.vq[ub][0][q] * s.vq[we][1][q] + s.vq[ub1][0][q] * s.vq[we][2][q];
            cv = fmaf(tb.T3[a][b][e], term, cv);
          }
        }
        val = fmaf(dt * conv, cv, val);
        gx = dt * nu * gx + (c == 0 ? dt * pw : 0.f);
        gy = dt * nu * gy + (c == 1 ? dt * pw : 0.f);
        s.cv[c * d::NT + a][0][q] = om * val;
        s.cv[c * d::NT + a][1][q] = om * gx * ih;
        s.cv[c * d::NT + a][2][q] = om * gy * ih;
      }
    }
  }
  __syncwarp();
  for (int it = lane; it < 2 * d::NT * d::NVL * d::NQ; it += 32) {
    const int f = it / (d::NVL * d::NQ), r = it % (d::NVL * d::NQ);
    const int j = r / d::NQ, qx = r % d::NQ;
    float a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int qy = 0; qy < d::NQ; ++qy) {
      const int q = qy * d::NQ + qx;
      a1 = fmaf(tb.Bv[qy][j], s.cv[f][0][q], a1);
      a1 = fmaf(tb.Dv[qy][j], s.cv[f][2][q], a1);
      a2 = fmaf(tb.Bv[qy][j], s.cv[f][1][q], a2);
    }
    s.t1[f][0][j][qx] = a1;
    s.t1[f][1][j][qx] = a2;
  }
  __syncwarp();
  for (int it = lane; it < 2 * d::NT * d::NVE; it += 32) {
    const int f = it / d::NVE, l = it % d::NVE;
    const int c = f / d::NT, a = f % d::NT;
    const int j = l / d::NVL, i = l % d::NVL;
    float v = 0.f;
#pragma unroll
    for (int qx = 0; qx < d::NQ; ++qx) {
      v = fmaf(tb.Bv[qx][i], s.t1[f][0][j][qx], v);
      v = fmaf(tb.Dv[qx][i], s.t1[f][1][j][qx], v);
    }
    s.out[a * (2 * d::NVE + d::NPE) + c * d::NVE + l] = v;
  }
  for (int it = lane; it < d::NT * d::NPE; it += 32) {
    const int a = it / d::NPE, l = it % d::NPE;
    const int j = l / d::NPL, i = l % d::NPL;
    float v = 0.f;
    for (int qy = 0; qy < d::NQ; ++qy)
      for (int qx = 0; qx < d::NQ; ++qx) v = fmaf(tb.Bp[qy][j] * tb.Bp[qx][i], s.cp[a][qy * d::NQ + qx], v);
    s.out[a * (2 * d::NVE + d::NPE) + 2 * d::NVE + l] = v;
  }
  __syncwarp();
  double* dst = ye + ((int64_t)slab * g.ncells() + cell) * d::ELEM;
  for (int it = lane; it < d::ELEM; it += 32) dst[it] = (double)s.out[it];
}

template <int K, int Q>
__global__ void __launch_bounds__(32 * kWarps)
element_f32_kernel(LevelGeom g, FeTables T, PhysParams ph, const double* __restrict__ W,
                   const double* __restrict__ x, double* __restrict__ ye) {
  __shared__ TabF<K, Q> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tab_f<K, Q>(T, tb);
  __syncthreads();
  const int cell = blockIdx.x * kWarps + threadIdx.x / 32;
  if (cell >= g.ncells()) return;
  element_body_f32<K, Q>(g, tb, ph, W, x, ye, reinterpret_cast<ElemSmemF<K, Q>*>(smem_raw)[threadIdx.x / 32], cell,
                         blockIdx.y);
}

// Batched FP32 Jacobian: one CTA per (member, group of kWarps cells, slab).
template <int K, int Q>
__global__ void __launch_bounds__(32 * kWarps)
bt_element_f32_kernel(const BatchSeg* __restrict__ segs, int nseg, FeTables T, const double* __restrict__ x,
                      double* __restrict__ ye) {
  __shared__ TabF<K, Q> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_tab_f<K, Q>(T, tb);
  __syncthreads();
  const int m = batch_find<BU_ELEM>(segs, nseg, blockIdx.x);
  const LevelGeom g = segs[m].g;
  const int cb = (g.ncells() + kWarps - 1) / kWarps;
  const int64_t local = blockIdx.x - segs[m].u_elem;
  const int slab = (int)(local / cb), cell = (int)(local % cb) * kWarps + threadIdx.x / 32;
  if (cell >= g.ncells()) return;
  element_body_f32<K, Q>(g, tb, segs[m].ph, segs[m].W, x + segs[m].off, ye + segs[m].off_ye,
                         reinterpret_cast<ElemSmemF<K, Q>*>(smem_raw)[threadIdx.x / 32], cell, slab);
}

// The reference tables are copied once per CTA into shared memory: element_body
// indexes them with lane-dependent indices, which kernel-parameter space serves one
// address at a time.  T is a grid constant, so its address is taken without a copy.
__device__ __forceinline__ void stage_fe_tables(const FeTables& T, FeTables& Ts) {
  const double* src = reinterpret_cast<const double*>(&T);
  double* dst = reinterpret_cast<double*>(&Ts);
  for (int i = threadIdx.x; i < (int)(sizeof(FeTables) / sizeof(double)); i += blockDim.x) dst[i] = src[i];
}

template <int K, int Q, bool LIN>
__global__ void __launch_bounds__(32 * kWarps)
element_kernel(LevelGeom g, const __grid_constant__ FeTables T, PhysParams ph, const double* __restrict__ W,
               const double* __restrict__ x, double* __restrict__ ye) {
  __shared__ FeTables Ts;
  stage_fe_tables(T, Ts);
  __syncthreads();
  const int cell = blockIdx.x * kWarps + threadIdx.x / 32;
  if (cell >= g.ncells()) return;
  element_body<K, Q, LIN>(g, Ts, ph, W, x, ye, cell, blockIdx.y);
}

// Batched: one CTA per (member, group of kWarps cells, slab); x and ye are arenas.
template <int K, int Q, bool LIN>
__global__ void __launch_bounds__(32 * kWarps)
bt_element_kernel(const BatchSeg* __restrict__ segs, int nseg, const __grid_constant__ FeTables T,
                  const double* __restrict__ x, double* __restrict__ ye) {
  __shared__ FeTables Ts;
  stage_fe_tables(T, Ts);
  __syncthreads();
  const int m = batch_find<BU_ELEM>(segs, nseg, blockIdx.x);
  const LevelGeom g = segs[m].g;
  const PhysParams ph = segs[m].ph;
  const int cb = (g.ncells() + kWarps - 1) / kWarps;
  const int64_t lu = blockIdx.x - segs[m].u_elem;
  const int slab = (int)(lu / cb);
  const int cell = (int)(lu % cb) * kWarps + threadIdx.x / 32;
  if (cell >= g.ncells()) return;
  element_body<K, Q, LIN>(g, Ts, ph, segs[m].W, x + segs[m].off, ye + segs[m].off_ye, cell, slab);
}

// Sums element contributions into the global vector (fixed cell order) and sets
// the Dirichlet rows: y = x for J, y = U - g for F.
template <int K, int Q, bool LIN>
__device__ __forceinline__ void assemble_body(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                                              const double* __restrict__ ye, const double* __restrict__ x,
                                              double* __restrict__ y, int64_t idx) {
  using d = D<K, Q>;
  const int S = g.S, nv = g.nv, np = g.np;
  const int64_t blk = idx / S;
  const int sp = int(idx % S);
  const int slab = int(blk / d::NT), a = int(blk % d::NT);
  const int nv2 = nv * nv;
  const int64_t base = (int64_t)slab * g.ncells();
  double acc = 0.0;
  if (sp < 2 * nv2) {
    const int c = sp / nv2, t = sp % nv2;
    const int gx = t % nv, gy = t / nv;
    if (vel_dirichlet(g, gx, gy)) {
      if (LIN) {
        y[idx] = x[idx];
      } else {
        double ux, uy;
        dirichlet_velocity(ph, gx, gy, nv, g.h / (K + 1), ph.t0 + (slab + T.tnode[a]) * g.dt, ux, uy);
        y[idx] = x[idx] - (c == 0 ? ux : uy);
      }
      return;
    }
    const int p = K + 1;
    const int cx0 = (gx - 1) / p, cx1 = min(gx / p, g.n - 1);
    const int cy0 = (gy - 1) / p, cy1 = min(gy / p, g.n - 1);
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int l = (gy - cy * p) * d::NVL + (gx - cx * p);
        acc += ye[(base + cy * g.n + cx) * d::ELEM + a * (2 * d::NVE + d::NPE) + c * d::NVE + l];
      }
  } else {
    const int t = sp - 2 * nv2;
    const int px = t % np, py = t / np;
    const int p = K;
    const int cx0 = px == 0 ? 0 : (px - 1) / p, cx1 = min(px / p, g.n - 1);
    const int cy0 = py == 0 ? 0 : (py - 1) / p, cy1 = min(py / p, g.n - 1);
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int l = (py - cy * p) * d::NPL + (px - cx * p);
        acc += ye[(base + cy * g.n + cx) * d::ELEM + a * (2 * d::NVE + d::NPE) + 2 * d::NVE + l];
      }
  }
  y[idx] = acc;
}

template <int K, int Q, bool LIN>
__global__ void assemble_kernel(LevelGeom g, FeTables T, PhysParams ph, const double* __restrict__ ye,
                                const double* __restrict__ x, double* __restrict__ y) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  assemble_body<K, Q, LIN>(g, T, ph, ye, x, y, idx);
}

template <int K, int Q, bool LIN>
__global__ void bt_assemble_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, FeTables T,
                                   const double* __restrict__ ye, const double* __restrict__ x,
                                   double* __restrict__ y) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const LevelGeom g = segs[m].g;
  const int64_t off = segs[m].off;
  assemble_body<K, Q, LIN>(g, T, segs[m].ph, ye + segs[m].off_ye, x + off, y + off, u - segs[m].u_dof);
}

__device__ __forceinline__ void boundary_body(const LevelGeom& g, const FeTables& T, const PhysParams& ph,
                                              double* __restrict__ U, int64_t idx) {
  const int S = g.S, nv = g.nv, nv2 = nv * nv;
  const int64_t blk = idx / S;
  const int sp = int(idx % S);
  const int slab = int(blk / g.nt), a = int(blk % g.nt);
  double v = 0.0;
  if (sp < 2 * nv2) {
    const int c = sp / nv2, t = sp % nv2;
    const int gx = t % nv, gy = t / nv;
    if (vel_dirichlet(g, gx, gy)) {
      double ux, uy;
      dirichlet_velocity(ph, gx, gy, nv, g.h / (g.k + 1), ph.t0 + (slab + T.tnode[a]) * g.dt, ux, uy);
      v = c == 0 ? ux : uy;
    }
  }
  U[idx] = v;
}

__global__ void boundary_kernel(LevelGeom g, FeTables T, PhysParams ph, double* __restrict__ U) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= g.ndofs) return;
  boundary_body(g, T, ph, U, idx);
}

__global__ void bt_boundary_kernel(const BatchSeg* __restrict__ segs, int nseg, int64_t dofs, FeTables T,
                                   double* __restrict__ U) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= dofs) return;
  const int m = batch_find<BU_DOF>(segs, nseg, u);
  const LevelGeom g = segs[m].g;
  boundary_body(g, T, segs[m].ph, U + segs[m].off, u - segs[m].u_dof);
}

// Element convection matrices about W (per time DoF e of W):
//   Ce[slab][cell][e][c*2+d][i][j] = int phi_i [ delta_cd (W_e.grad) phi_j + phi_j d_d W_{e,c} ]
// One warp per (cell, slab).  W and its gradient are interpolated to the Gauss
// points by sum factorisation; the matrices are sum-factorised too: with
// phi_i = b_ix(x) b_iy(y) every integrand is a weight product in x times one in y
// times a field F at the quadrature point, so the x sums come first,
//   P_F[ix][jx][qy] = sum_qx w_qx b_ix(qx) c_jx(qx) F(qx, qy)   (c = b', or b),
// and each entry is then a sum over qy (NQ terms instead of NQ^2 per entry).
// CT is the arithmetic and storage type: double for the FP64 factorisation, float
// for the FP32/BF16 ones (whose blocks are assembled in FP32).
template <int K, int Q, typename CT>
__global__ void __launch_bounds__(32 * kWarps)
conv_elements_kernel(LevelGeom g, FeTables T, const double* __restrict__ W, CT* __restrict__ Ce) {
  using d = D<K, Q>;
  constexpr int NT = d::NT, NVL = d::NVL, NQ = d::NQ, NVE = d::NVE, NQ2 = d::NQ2;
  struct Sm {
    CT wn[2 * NT][NVE];
    CT t1[2 * NT][2][NVL][NQ];
    CT wq[2 * NT][3][NQ2];
    CT P[6][NVL][NVL][NQ];
  };
  __shared__ CT bv[NQ][NVL], dv[NQ][NVL];
  __shared__ CT ww[2][NVL][NVL][NQ];  // w_q b_i(q) b'_j(q) and w_q b_i(q) b_j(q)
  for (int e = threadIdx.x; e < NQ * NVL; e += blockDim.x) {
    const int q = e / NVL, i = e % NVL;
    bv[q][i] = (CT)T.Bv[q][i];
    dv[q][i] = (CT)T.Dv[q][i];
  }
  for (int e = threadIdx.x; e < NVL * NVL * NQ; e += blockDim.x) {
    const int i = e / (NVL * NQ), j = (e / NQ) % NVL, q = e % NQ;
    ww[0][i][j][q] = (CT)(T.wq[q] * T.Bv[q][i] * T.Dv[q][j]);
    ww[1][i][j][q] = (CT)(T.wq[q] * T.Bv[q][i] * T.Bv[q][j]);
  }
  __syncthreads();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& s = reinterpret_cast<Sm*>(smem_raw)[threadIdx.x / 32];
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kWarps + threadIdx.x / 32;
  const int slab = blockIdx.y;
  if (cell >= g.ncells()) return;
  const int CI = cell % g.n, CJ = cell / g.n;
  const int nv = g.nv;
  const int64_t nv2 = (int64_t)nv * nv;
  const CT h = (CT)g.h, ih = (CT)(1.0 / g.h);
  for (int it = lane; it < 2 * NT * NVE; it += 32) {
    const int f = it / NVE, l = it % NVE;  // f = c*NT + e
    const int c = f / NT, e = f % NT;
    const int gx = CI * (K + 1) + l % NVL, gy = CJ * (K + 1) + l / NVL;
    s.wn[f][l] = (CT)W[((int64_t)slab * NT + e) * g.S + c * nv2 + (int64_t)gy * nv + gx];
  }
  __syncwarp();
  for (int it = lane; it < 2 * NT * NVL * NQ; it += 32) {
    const int f = it / (NVL * NQ), r = it % (NVL * NQ);
    const int j = r / NQ, qx = r % NQ;
    CT v = 0, dvv = 0;
    for (int i = 0; i < NVL; ++i) {
      v = fma(bv[qx][i], s.wn[f][j * NVL + i], v);
      dvv = fma(dv[qx][i], s.wn[f][j * NVL + i], dvv);
    }
    s.t1[f][0][j][qx] = v;
    s.t1[f][1][j][qx] = dvv;
  }
  __syncwarp();
  for (int it = lane; it < 2 * NT * NQ2; it += 32) {
    const int f = it / NQ2, q = it % NQ2;
    const int qy = q / NQ, qx = q % NQ;
    CT v = 0, vx = 0, vy = 0;
    for (int j = 0; j < NVL; ++j) {
      v = fma(bv[qy][j], s.t1[f][0][j][qx], v);
      vx = fma(bv[qy][j], s.t1[f][1][j][qx], vx);
      vy = fma(dv[qy][j], s.t1[f][0][j][qx], vy);
    }
    s.wq[f][0][q] = v;
    s.wq[f][1][q] = vx * ih;
    s.wq[f][2][q] = vy * ih;
  }
  __syncwarp();
  CT* dst = Ce + ((int64_t)slab * g.ncells() + cell) * (NT * 4 * NVE * NVE);
  for (int e = 0; e < NT; ++e) {
    // x sums; fields: 0 W_x (against b'_jx), 1 W_y, 2 d_x W_x, 3 d_y W_x, 4 d_x W_y, 5 d_y W_y
    for (int it = lane; it < 6 * NVL * NVL * NQ; it += 32) {
      const int f = it / (NVL * NVL * NQ), r = it % (NVL * NVL * NQ);
      const int ix = r / (NVL * NQ), jx = (r / NQ) % NVL, qy = r % NQ;
      const int c = f == 0 ? 0 : f == 1 ? 1 : (f - 2) / 2;
      const int comp = f < 2 ? 0 : 1 + (f - 2) % 2;
      const CT* fld = &s.wq[c * NT + e][comp][qy * NQ];
      const CT* wt = &ww[f == 0 ? 0 : 1][ix][jx][0];
      CT acc = 0;
#pragma unroll
      for (int qx = 0; qx < NQ; ++qx) acc = fma(wt[qx], fld[qx], acc);
      s.P[f][ix][jx][qy] = acc;
    }
    __syncwarp();
    CT* m = dst + (int64_t)e * 4 * NVE * NVE;
    for (int it = lane; it < NVE * NVE; it += 32) {
      const int i = it / NVE, j = it % NVE;
      const int iy = i / NVL, ix = i % NVL, jy = j / NVL, jx = j % NVL;
      CT adv = 0, b00 = 0, b01 = 0, b10 = 0, b11 = 0;
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy) {
        const CT wb = ww[1][iy][jy][qy], wd = ww[0][iy][jy][qy];
        adv = fma(wb, s.P[0][ix][jx][qy], fma(wd, s.P[1][ix][jx][qy], adv));
        b00 = fma(wb, s.P[2][ix][jx][qy], b00);
        b01 = fma(wb, s.P[3][ix][jx][qy], b01);
        b10 = fma(wb, s.P[4][ix][jx][qy], b10);
        b11 = fma(wb, s.P[5][ix][jx][qy], b11);
      }
      // cell weights: h^2 for the area, 1/h for the derivative of phi_j in the advection
      adv *= h;
      const CT h2 = h * h;
      m[0 * NVE * NVE + it] = adv + h2 * b00;
      m[1 * NVE * NVE + it] = h2 * b01;
      m[2 * NVE * NVE + it] = h2 * b10;
      m[3 * NVE * NVE + it] = adv + h2 * b11;
    }
    __syncwarp();
  }
}

__global__ void inject_kernel(LevelGeom gf, LevelGeom gc, const double* __restrict__ Wf, double* __restrict__ Wc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= gc.ndofs) return;
  const int64_t blk = idx / gc.S;
  const int sp = int(idx % gc.S);
  const int nvc2 = gc.nv * gc.nv;
  int64_t src;
  if (sp < 2 * nvc2) {
    const int c = sp / nvc2, t = sp % nvc2;
    const int x = t % gc.nv, y = t / gc.nv;
    src = c * (int64_t)gf.nv * gf.nv + (int64_t)(2 * y) * gf.nv + 2 * x;
  } else {
    const int t = sp - 2 * nvc2;
    const int x = t % gc.np, y = t / gc.np;
    src = 2 * (int64_t)gf.nv * gf.nv + (int64_t)(2 * y) * gf.np + 2 * x;
  }
  Wc[idx] = Wf[blk * gf.S + src];
}

template <int K, int Q, bool LIN>
void run_element(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W, const double* x,
                 double* y, double* ye, cudaStream_t s) {
  const size_t smem = sizeof(ElemSmem<K, Q, LIN>) * kWarps;
  auto kern = element_kernel<K, Q, LIN>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((g.ncells() + kWarps - 1) / kWarps, g.N);
  kern<<<grid, 32 * kWarps, smem, s>>>(g, T, ph, W, x, ye);
  WR_LAUNCH_CHECK();
  const int threads = 256;
  assemble_kernel<K, Q, LIN><<<(unsigned)((g.ndofs + threads - 1) / threads), threads, 0, s>>>(g, T, ph, ye, x, y);
  WR_LAUNCH_CHECK();
}

template <bool LIN>
void dispatch_element(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W, const double* x,
                      double* y, double* ye, cudaStream_t s) {
  if (g.k == 1 && g.q == 0) run_element<1, 0, LIN>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 1 && g.q == 1) run_element<1, 1, LIN>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 2 && g.q == 0) run_element<2, 0, LIN>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 2 && g.q == 1) run_element<2, 1, LIN>(g, T, ph, W, x, y, ye, s);
  else if constexpr (!LIN) {  // the residual with DG(2), DG(3) (their J is launch_jacobian_wq)
    if (g.k == 1 && g.q == 2) run_element<1, 2, false>(g, T, ph, W, x, y, ye, s);
    else if (g.k == 1 && g.q == 3) run_element<1, 3, false>(g, T, ph, W, x, y, ye, s);
    else if (g.k == 2 && g.q == 2) run_element<2, 2, false>(g, T, ph, W, x, y, ye, s);
    else if (g.k == 2 && g.q == 3) run_element<2, 3, false>(g, T, ph, W, x, y, ye, s);
    else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
  } else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

template <int K, int Q, typename CT>
void run_conv(const LevelGeom& g, const FeTables& T, const double* W, CT* Ce, cudaStream_t s) {
  using d = D<K, Q>;
  const size_t smem = sizeof(CT) * (2 * d::NT * d::NVE + 2 * d::NT * 2 * d::NVL * d::NQ + 2 * d::NT * 3 * d::NQ2 +
                                    6 * d::NVL * d::NVL * d::NQ) * kWarps;
  auto kern = conv_elements_kernel<K, Q, CT>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((g.ncells() + kWarps - 1) / kWarps, g.N);
  kern<<<grid, 32 * kWarps, smem, s>>>(g, T, W, Ce);
  WR_LAUNCH_CHECK();
}

template <int K, int Q, bool LIN>
void run_bt_element(const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T, const double* x,
                    double* y, double* ye, cudaStream_t s) {
  const size_t smem = sizeof(ElemSmem<K, Q, LIN>) * kWarps;
  auto kern = bt_element_kernel<K, Q, LIN>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (units > 0) {
    kern<<<(unsigned)units, 32 * kWarps, smem, s>>>(segs, nseg, T, x, ye);
    WR_LAUNCH_CHECK();
  }
  if (dofs > 0) {
    bt_assemble_kernel<K, Q, LIN><<<(unsigned)((dofs + 255) / 256), 256, 0, s>>>(segs, nseg, dofs, T, ye, x, y);
    WR_LAUNCH_CHECK();
  }
}

template <int K, int Q>
void run_element_f32(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W, const double* x,
                     double* y, double* ye, cudaStream_t s) {
  const size_t smem = sizeof(ElemSmemF<K, Q>) * kWarps;
  auto kern = element_f32_kernel<K, Q>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((g.ncells() + kWarps - 1) / kWarps, g.N);
  kern<<<grid, 32 * kWarps, smem, s>>>(g, T, ph, W, x, ye);
  WR_LAUNCH_CHECK();
  assemble_kernel<K, Q, true><<<(unsigned)((g.ndofs + 255) / 256), 256, 0, s>>>(g, T, ph, ye, x, y);
  WR_LAUNCH_CHECK();
}

template <int K, int Q>
void run_bt_element_f32(const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                        const double* x, double* y, double* ye, cudaStream_t s) {
  const size_t smem = sizeof(ElemSmemF<K, Q>) * kWarps;
  auto kern = bt_element_f32_kernel<K, Q>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (units > 0) {
    kern<<<(unsigned)units, 32 * kWarps, smem, s>>>(segs, nseg, T, x, ye);
    WR_LAUNCH_CHECK();
  }
  if (dofs > 0) {
    bt_assemble_kernel<K, Q, true><<<(unsigned)((dofs + 255) / 256), 256, 0, s>>>(segs, nseg, dofs, T, ye, x, y);
    WR_LAUNCH_CHECK();
  }
}

// ---------------------------------------------------------------- J(W) x of the solver
// The Jacobian action every Chebyshev residual, restricted residual and FGMRES
// iteration applies.  Same weak form and quadrature as element_body<.., true>, laid out
// for the FP64 pipe, which bounds it on GB300 (FP64 at 1/64 of the FP32 rate):
//  * W, grad W at the Gauss points do not change between linearisations: wq_kernel
//    tabulates them once per linearisation (reference-cell gradients), so an apply
//    interpolates only x;
//  * every constant factor is folded into per-level tables: the quadrature weights into
//    the test-function tables, h, dt, nu and conv into the temporal matrices
//    (h^2 Kt, h^2 tau(0), dt conv h T3, dt nu Wt, dt h Wt), so the pointwise stage has
//    no scaling multiplications and gradients stay in reference coordinates;
//  * the convection is formed once per (b, e, c) and contracted with T3 afterwards;
//  * pressure interpolation and its test contraction are sum-factorised too, and the
//    jump value x^- needs no derivatives.
// Element results go to the same per-element buffer as element_body's, summed by
// assemble_kernel.
template <int K, int Q>
struct JacTab {
  using d = D<K, Q>;
  double Bv[d::NQ][d::NVL], Dv[d::NQ][d::NVL], Bp[d::NQ][d::NPL];     // interpolation
  double BvW[d::NQ][d::NVL], DvW[d::NQ][d::NVL], BpW[d::NQ][d::NPL];  // test functions x Gauss weight
  double KtH[d::NT][d::NT], tauH[d::NT], T3H[d::NT][d::NT][d::NT], WtN[d::NT][d::NT], WtP[d::NT][d::NT];
};

template <int K, int Q>
__device__ __forceinline__ void build_jac_tab(const FeTables& T, const LevelGeom& g, const PhysParams& ph,
                                              JacTab<K, Q>& tb) {
  using d = D<K, Q>;
  const double h = g.h, dt = g.dt;
  for (int e = threadIdx.x; e < d::NQ * d::NVL; e += blockDim.x) {
    const int q = e / d::NVL, i = e % d::NVL;
    tb.Bv[q][i] = T.Bv[q][i];
    tb.Dv[q][i] = T.Dv[q][i];
    tb.BvW[q][i] = T.wq[q] * T.Bv[q][i];
    tb.DvW[q][i] = T.wq[q] * T.Dv[q][i];
  }
  for (int e = threadIdx.x; e < d::NQ * d::NPL; e += blockDim.x) {
    const int q = e / d::NPL, i = e % d::NPL;
    tb.Bp[q][i] = T.Bp[q][i];
    tb.BpW[q][i] = T.wq[q] * T.Bp[q][i];
  }
  for (int e = threadIdx.x; e < d::NT * d::NT * d::NT; e += blockDim.x) {
    const int a = e / (d::NT * d::NT), b = (e / d::NT) % d::NT, c = e % d::NT;
    tb.T3H[a][b][c] = dt * ph.conv * h * T.T3[a][b][c];
    if (c == 0) {
      tb.KtH[a][b] = h * h * T.Kt[a][b];
      tb.WtN[a][b] = dt * ph.nu * T.Wt[a][b];
      tb.WtP[a][b] = dt * h * T.Wt[a][b];
    }
  }
  for (int e = threadIdx.x; e < d::NT; e += blockDim.x) tb.tauH[e] = h * h * T.tau0[e];
}

// Per (cell, slab): W_{c,b} and its reference-cell gradient at the Gauss points,
// field (c NT + b) 3 + {value, d/dx, d/dy}, Gauss point fastest.
template <int K, int Q>
struct JacSmem {
  using d = D<K, Q>;
  static constexpr int NF = 2 * d::NT;      // velocity fields (component c, temporal DoF b)
  double vn[NF][d::NVE];                    // nodal x (W in wq_kernel)
  double mn[2][d::NVE];                     // nodal x^-: the previous slab's last temporal DoF
  double pn[d::NT][d::NPE];
  double t1[NF][2][d::NVL][d::NQ];          // x pass (value, d/dx); then the test y pass
  double tm[2][d::NVL][d::NQ];
  double tp[d::NT][d::NPL][d::NQ];          // x pass of the pressure; then its test y pass
  double vq[NF][3][d::NQ2];                 // value, d/dx, d/dy; overwritten by the coefficients
  double mq[2][d::NQ2];
  double pq[d::NT][d::NQ2];                 // pressure; overwritten by the divergence coefficient
  double out[d::ELEM];
};

template <int K, int Q>
__global__ void __launch_bounds__(32 * kWarps)
wq_kernel(LevelGeom g, const __grid_constant__ FeTables T, const double* __restrict__ W, double* __restrict__ Wq) {
  using d = D<K, Q>;
  using SM = JacSmem<K, Q>;
  constexpr int NF = SM::NF;
  __shared__ FeTables Ts;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_fe_tables(T, Ts);
  __syncthreads();
  const int cell = blockIdx.x * kWarps + threadIdx.x / 32, slab = blockIdx.y;
  if (cell >= g.ncells()) return;
  SM& s = reinterpret_cast<SM*>(smem_raw)[threadIdx.x / 32];
  const int lane = threadIdx.x & 31;
  const int CI = cell % g.n, CJ = cell / g.n;
  const int64_t nv2 = (int64_t)g.nv * g.nv;
  for (int it = lane; it < NF * d::NVE; it += 32) {
    const int f = it / d::NVE, l = it % d::NVE, c = f / d::NT, b = f % d::NT;
    const int gx = CI * (K + 1) + l % d::NVL, gy = CJ * (K + 1) + l / d::NVL;
    s.vn[f][l] = W[((int64_t)slab * d::NT + b) * g.S + c * nv2 + (int64_t)gy * g.nv + gx];
  }
  __syncwarp();
  for (int it = lane; it < NF * d::NVL * d::NQ; it += 32) {
    const int f = it / (d::NVL * d::NQ), r = it % (d::NVL * d::NQ), j = r / d::NQ, qx = r % d::NQ;
    double v = 0.0, dv = 0.0;
#pragma unroll
    for (int i = 0; i < d::NVL; ++i) {
      v = fma(Ts.Bv[qx][i], s.vn[f][j * d::NVL + i], v);
      dv = fma(Ts.Dv[qx][i], s.vn[f][j * d::NVL + i], dv);
    }
    s.t1[f][0][j][qx] = v;
    s.t1[f][1][j][qx] = dv;
  }
  __syncwarp();
  double* dst = Wq + ((int64_t)slab * g.ncells() + cell) * (NF * 3 * d::NQ2);
  for (int it = lane; it < NF * d::NQ2; it += 32) {
    const int f = it / d::NQ2, q = it % d::NQ2, qy = q / d::NQ, qx = q % d::NQ;
    double v = 0.0, vx = 0.0, vy = 0.0;
#pragma unroll
    for (int j = 0; j < d::NVL; ++j) {
      v = fma(Ts.Bv[qy][j], s.t1[f][0][j][qx], v);
      vx = fma(Ts.Bv[qy][j], s.t1[f][1][j][qx], vx);
      vy = fma(Ts.Dv[qy][j], s.t1[f][0][j][qx], vy);
    }
    dst[(f * 3 + 0) * d::NQ2 + q] = v;
    dst[(f * 3 + 1) * d::NQ2 + q] = vx;
    dst[(f * 3 + 2) * d::NQ2 + q] = vy;
  }
}

// Elements per warp of jac_kernel (cells cell0 .. cell0+E-1 of one slab).  Q3/Q2 DG(0)
// and DG(1) take two elements (stages of 25 Gauss points and 30 to 100 interpolation
// items per element fill 32-lane warps better in pairs; 6.6 KB per element leaves 16
// warps per SM), DG(2) and DG(3) one.  Q2/Q1 has 16 Gauss points and 8 to 72 items per
// stage: DG(0) and DG(1) take four elements (2.3 or 4 KB per element, 24 or 12 warps
// per SM), DG(2) and DG(3) two, so that their larger footprint and register count
// leave 8 to 12 warps per SM.
template <int K, int Q>
struct JacE {
  static constexpr int E = Q <= 1 ? (K == 2 ? 2 : 4) : (K == 2 ? 1 : 2);
};

// One warp: the element contributions of J(W) x on E cells (cell0 + e) of one slab.
// Every stage loop runs over the items of all E elements, so that short stages fill
// the warp; elements beyond the mesh are skipped.
template <int K, int Q, int E>
__device__ __forceinline__ void jac_body(const LevelGeom& g, const JacTab<K, Q>& tb, const double* __restrict__ Wq,
                                         const double* __restrict__ x, double* __restrict__ ye, JacSmem<K, Q>* s,
                                         int cell0, int slab) {
  using d = D<K, Q>;
  using SM = JacSmem<K, Q>;
  constexpr int NF = SM::NF, NT = d::NT, NVL = d::NVL, NPL = d::NPL, NQ = d::NQ, NQ2 = d::NQ2;
  const int lane = threadIdx.x & 31;
  const int S = g.S, nc = g.ncells();
  const int nin = E == 1 ? 1 : min(E, nc - cell0);  // elements of this warp inside the mesh
  constexpr int ne = E;  // every stage runs all E elements; those beyond the mesh see zero input
  const int64_t nv2 = (int64_t)g.nv * g.nv;

  // ---- gather x (Dirichlet velocity rows of J are the identity, set by the assembly)
  for (int it = lane; it < ne * 2 * d::NVE; it += 32) {
    const int e = E == 1 ? 0 : it / (2 * d::NVE), r = E == 1 ? it : it % (2 * d::NVE), c = r / d::NVE, l = r % d::NVE;
    const int cell = min(cell0 + e, nc - 1), CI = cell % g.n, CJ = cell / g.n;
    const int gx = CI * (K + 1) + l % NVL, gy = CJ * (K + 1) + l / NVL;
    const int64_t sp = c * nv2 + (int64_t)gy * g.nv + gx;
    const bool dir = vel_dirichlet(g, gx, gy) || e >= nin;
#pragma unroll
    for (int b = 0; b < NT; ++b) s[e].vn[c * NT + b][l] = dir ? 0.0 : x[((int64_t)slab * NT + b) * S + sp];
    s[e].mn[c][l] = (slab > 0 && !dir) ? x[((int64_t)(slab - 1) * NT + (NT - 1)) * S + sp] : 0.0;
  }
  for (int it = lane; it < ne * NT * d::NPE; it += 32) {
    const int e = E == 1 ? 0 : it / (NT * d::NPE), r = E == 1 ? it : it % (NT * d::NPE), b = r / d::NPE, l = r % d::NPE;
    const int cell = min(cell0 + e, nc - 1), CI = cell % g.n, CJ = cell / g.n;
    const int px = CI * K + l % NPL, py = CJ * K + l / NPL;
    s[e].pn[b][l] = e < nin ? x[((int64_t)slab * NT + b) * S + 2 * nv2 + (int64_t)py * g.np + px] : 0.0;
  }
  __syncwarp();

  // ---- interpolation to the Gauss points, x pass
  for (int it = lane; it < ne * NF * NVL * NQ; it += 32) {
    const int e = E == 1 ? 0 : it / (NF * NVL * NQ), r0 = E == 1 ? it : it % (NF * NVL * NQ);
    const int f = r0 / (NVL * NQ), r = r0 % (NVL * NQ), j = r / NQ, qx = r % NQ;
    double v = 0.0, dv = 0.0;
#pragma unroll
    for (int i = 0; i < NVL; ++i) {
      v = fma(tb.Bv[qx][i], s[e].vn[f][j * NVL + i], v);
      dv = fma(tb.Dv[qx][i], s[e].vn[f][j * NVL + i], dv);
    }
    s[e].t1[f][0][j][qx] = v;
    s[e].t1[f][1][j][qx] = dv;
  }
  for (int it = lane; it < ne * 2 * NVL * NQ; it += 32) {
    const int e = E == 1 ? 0 : it / (2 * NVL * NQ), r0 = E == 1 ? it : it % (2 * NVL * NQ);
    const int c = r0 / (NVL * NQ), r = r0 % (NVL * NQ), j = r / NQ, qx = r % NQ;
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < NVL; ++i) v = fma(tb.Bv[qx][i], s[e].mn[c][j * NVL + i], v);
    s[e].tm[c][j][qx] = v;
  }
  for (int it = lane; it < ne * NT * NPL * NQ; it += 32) {
    const int e = E == 1 ? 0 : it / (NT * NPL * NQ), r0 = E == 1 ? it : it % (NT * NPL * NQ);
    const int b = r0 / (NPL * NQ), r = r0 % (NPL * NQ), j = r / NQ, qx = r % NQ;
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < NPL; ++i) v = fma(tb.Bp[qx][i], s[e].pn[b][j * NPL + i], v);
    s[e].tp[b][j][qx] = v;
  }
  __syncwarp();
  // y pass
  for (int it = lane; it < ne * NF * NQ2; it += 32) {
    const int e = E == 1 ? 0 : it / (NF * NQ2), r0 = E == 1 ? it : it % (NF * NQ2);
    const int f = r0 / NQ2, q = r0 % NQ2, qy = q / NQ, qx = q % NQ;
    double v = 0.0, vx = 0.0, vy = 0.0;
#pragma unroll
    for (int j = 0; j < NVL; ++j) {
      v = fma(tb.Bv[qy][j], s[e].t1[f][0][j][qx], v);
      vx = fma(tb.Bv[qy][j], s[e].t1[f][1][j][qx], vx);
      vy = fma(tb.Dv[qy][j], s[e].t1[f][0][j][qx], vy);
    }
    s[e].vq[f][0][q] = v;
    s[e].vq[f][1][q] = vx;
    s[e].vq[f][2][q] = vy;
  }
  for (int it = lane; it < ne * 2 * NQ2; it += 32) {
    const int e = E == 1 ? 0 : it / (2 * NQ2), r0 = E == 1 ? it : it % (2 * NQ2), c = r0 / NQ2, q = r0 % NQ2, qy = q / NQ, qx = q % NQ;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < NVL; ++j) v = fma(tb.Bv[qy][j], s[e].tm[c][j][qx], v);
    s[e].mq[c][q] = v;
  }
  for (int it = lane; it < ne * NT * NQ2; it += 32) {
    const int e = E == 1 ? 0 : it / (NT * NQ2), r0 = E == 1 ? it : it % (NT * NQ2), b = r0 / NQ2, q = r0 % NQ2, qy = q / NQ, qx = q % NQ;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < NPL; ++j) v = fma(tb.Bp[qy][j], s[e].tp[b][j][qx], v);
    s[e].pq[b][q] = v;
  }
  __syncwarp();

  // ---- pointwise coefficients (each lane reads and overwrites its own Gauss point)
  for (int it = lane; it < ne * NQ2; it += 32) {
    const int e = E == 1 ? 0 : it / NQ2, q = E == 1 ? it : it % NQ2;
    SM& se = s[e];
    const double* __restrict__ wq = Wq + ((int64_t)slab * nc + min(cell0 + e, nc - 1)) * (NF * 3 * NQ2) + q;
    double Wv[NF][3], X[NF][3], p[NT], dv[NT], xm[2];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Wv[f][k] = wq[(f * 3 + k) * NQ2];
        X[f][k] = se.vq[f][k][q];
      }
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      p[b] = se.pq[b][q];
      dv[b] = X[0 * NT + b][1] + X[1 * NT + b][2];
    }
    xm[0] = se.mq[0][q];
    xm[1] = se.mq[1][q];
    // Newton convection (W_b . grad) x_{c,e} + (x_b . grad) W_{c,e}, per (b, e, c)
    double P[NT][NT][2];
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int ee = 0; ee < NT; ++ee)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int fe = c * NT + ee;
          double t = Wv[0 * NT + b][0] * X[fe][1];
          t = fma(Wv[1 * NT + b][0], X[fe][2], t);
          t = fma(X[0 * NT + b][0], Wv[fe][1], t);
          P[b][ee][c] = fma(X[1 * NT + b][0], Wv[fe][2], t);
        }
#pragma unroll
    for (int a = 0; a < NT; ++a) {
      double pw = 0.0, dw = 0.0;
#pragma unroll
      for (int b = 0; b < NT; ++b) {
        pw = fma(tb.WtP[a][b], p[b], pw);
        dw = fma(tb.WtP[a][b], dv[b], dw);
      }
      se.pq[a][q] = dw;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        double val = -tb.tauH[a] * xm[c];
        double gx = c == 0 ? pw : 0.0, gy = c == 1 ? pw : 0.0;
#pragma unroll
        for (int b = 0; b < NT; ++b) {
          val = fma(tb.KtH[a][b], X[c * NT + b][0], val);
          gx = fma(tb.WtN[a][b], X[c * NT + b][1], gx);
          gy = fma(tb.WtN[a][b], X[c * NT + b][2], gy);
#pragma unroll
          for (int ee = 0; ee < NT; ++ee) val = fma(tb.T3H[a][b][ee], P[b][ee][c], val);
        }
        se.vq[c * NT + a][0][q] = val;
        se.vq[c * NT + a][1][q] = gx;
        se.vq[c * NT + a][2][q] = gy;
      }
    }
  }
  __syncwarp();

  // ---- test contraction, y pass (weighted test tables)
  for (int it = lane; it < ne * NF * NVL * NQ; it += 32) {
    const int e = E == 1 ? 0 : it / (NF * NVL * NQ), r0 = E == 1 ? it : it % (NF * NVL * NQ);
    const int f = r0 / (NVL * NQ), r = r0 % (NVL * NQ), j = r / NQ, qx = r % NQ;
    double a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int qy = 0; qy < NQ; ++qy) {
      const int q = qy * NQ + qx;
      a1 = fma(tb.BvW[qy][j], s[e].vq[f][0][q], a1);
      a1 = fma(tb.DvW[qy][j], s[e].vq[f][2][q], a1);
      a2 = fma(tb.BvW[qy][j], s[e].vq[f][1][q], a2);
    }
    s[e].t1[f][0][j][qx] = a1;
    s[e].t1[f][1][j][qx] = a2;
  }
  for (int it = lane; it < ne * NT * NPL * NQ; it += 32) {
    const int e = E == 1 ? 0 : it / (NT * NPL * NQ), r0 = E == 1 ? it : it % (NT * NPL * NQ);
    const int a = r0 / (NPL * NQ), r = r0 % (NPL * NQ), j = r / NQ, qx = r % NQ;
    double v = 0.0;
#pragma unroll
    for (int qy = 0; qy < NQ; ++qy) v = fma(tb.BpW[qy][j], s[e].pq[a][qy * NQ + qx], v);
    s[e].tp[a][j][qx] = v;
  }
  __syncwarp();
  // x pass -> element output; layout a (2 NVE + NPE) + c NVE + l, then pressure
  for (int it = lane; it < ne * NF * d::NVE; it += 32) {
    const int e = E == 1 ? 0 : it / (NF * d::NVE), r0 = E == 1 ? it : it % (NF * d::NVE);
    const int f = r0 / d::NVE, l = r0 % d::NVE, c = f / NT, a = f % NT, j = l / NVL, i = l % NVL;
    double v = 0.0;
#pragma unroll
    for (int qx = 0; qx < NQ; ++qx) {
      v = fma(tb.BvW[qx][i], s[e].t1[f][0][j][qx], v);
      v = fma(tb.DvW[qx][i], s[e].t1[f][1][j][qx], v);
    }
    s[e].out[a * (2 * d::NVE + d::NPE) + c * d::NVE + l] = v;
  }
  for (int it = lane; it < ne * NT * d::NPE; it += 32) {
    const int e = E == 1 ? 0 : it / (NT * d::NPE), r0 = E == 1 ? it : it % (NT * d::NPE);
    const int a = r0 / d::NPE, l = r0 % d::NPE, j = l / NPL, i = l % NPL;
    double v = 0.0;
#pragma unroll
    for (int qx = 0; qx < NQ; ++qx) v = fma(tb.BpW[qx][i], s[e].tp[a][j][qx], v);
    s[e].out[a * (2 * d::NVE + d::NPE) + 2 * d::NVE + l] = v;
  }
  __syncwarp();
  double* dst = ye + ((int64_t)slab * g.ncells() + cell0) * d::ELEM;  // the E elements are consecutive
  for (int it = lane; it < nin * d::ELEM; it += 32) dst[it] = E == 1 ? s[0].out[it] : s[it / d::ELEM].out[it % d::ELEM];
}

template <int K, int Q>
__global__ void __launch_bounds__(32 * kWarps)
jac_kernel(LevelGeom g, const __grid_constant__ FeTables T, PhysParams ph, const double* __restrict__ Wq,
           const double* __restrict__ x, double* __restrict__ ye) {
  __shared__ JacTab<K, Q> tb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  build_jac_tab<K, Q>(T, g, ph, tb);
  __syncthreads();
  constexpr int E = JacE<K, Q>::E;
  const int cell0 = (blockIdx.x * kWarps + threadIdx.x / 32) * E;
  if (cell0 >= g.ncells()) return;
  jac_body<K, Q, E>(g, tb, Wq, x, ye, reinterpret_cast<JacSmem<K, Q>*>(smem_raw) + (threadIdx.x / 32) * E, cell0,
                    blockIdx.y);
}

template <int K, int Q>
void run_wq(const LevelGeom& g, const FeTables& T, const double* W, double* Wq, cudaStream_t s) {
  const size_t smem = sizeof(JacSmem<K, Q>) * kWarps;
  auto kern = wq_kernel<K, Q>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((g.ncells() + kWarps - 1) / kWarps, g.N);
  kern<<<grid, 32 * kWarps, smem, s>>>(g, T, W, Wq);
  WR_LAUNCH_CHECK();
}

template <int K, int Q>
void run_jac(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* Wq, const double* x,
             double* y, double* ye, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  constexpr int E = JacE<K, Q>::E;
  const size_t smem = sizeof(JacSmem<K, Q>) * kWarps * E;
  auto kern = jac_kernel<K, Q>;
  WR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((g.ncells() + kWarps * E - 1) / (kWarps * E), g.N);
  if (ev0) WR_CUDA(cudaEventRecord(ev0, s));
  kern<<<grid, 32 * kWarps, smem, s>>>(g, T, ph, Wq, x, ye);
  WR_LAUNCH_CHECK();
  if (ev1) WR_CUDA(cudaEventRecord(ev1, s));
  assemble_kernel<K, Q, true><<<(unsigned)((g.ndofs + 255) / 256), 256, 0, s>>>(g, T, ph, ye, x, y);
  WR_LAUNCH_CHECK();
}

template <bool LIN>
void dispatch_bt_element(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs,
                         const FeTables& T, const double* x, double* y, double* ye, cudaStream_t s) {
  if (k == 1 && q == 0) run_bt_element<1, 0, LIN>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 1 && q == 1) run_bt_element<1, 1, LIN>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 2 && q == 0) run_bt_element<2, 0, LIN>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 2 && q == 1) run_bt_element<2, 1, LIN>(segs, nseg, units, dofs, T, x, y, ye, s);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

}  // namespace

void bt_jacobian(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                 const double* x, double* y, double* ye, cudaStream_t s) {
  dispatch_bt_element<true>(k, q, segs, nseg, units, dofs, T, x, y, ye, s);
}

void bt_jacobian_f32(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                     const double* x, double* y, double* ye, cudaStream_t s) {
  if (k == 1 && q == 0) run_bt_element_f32<1, 0>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 1 && q == 1) run_bt_element_f32<1, 1>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 2 && q == 0) run_bt_element_f32<2, 0>(segs, nseg, units, dofs, T, x, y, ye, s);
  else if (k == 2 && q == 1) run_bt_element_f32<2, 1>(segs, nseg, units, dofs, T, x, y, ye, s);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

void bt_residual(int k, int q, const BatchSeg* segs, int nseg, int64_t units, int64_t dofs, const FeTables& T,
                 const double* U, double* F, double* ye, cudaStream_t s) {
  dispatch_bt_element<false>(k, q, segs, nseg, units, dofs, T, U, F, ye, s);
}

void bt_boundary(const BatchSeg* segs, int nseg, int64_t dofs, const FeTables& T, double* U, cudaStream_t s) {
  if (dofs <= 0) return;
  bt_boundary_kernel<<<(unsigned)((dofs + 255) / 256), 256, 0, s>>>(segs, nseg, dofs, T, U);
  WR_LAUNCH_CHECK();
}

void launch_residual(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* U, double* F,
                     double* ye, cudaStream_t s) {
  dispatch_element<false>(g, T, ph, nullptr, U, F, ye, s);
}

void launch_jacobian(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W, const double* x,
                     double* y, double* ye, cudaStream_t s) {
  dispatch_element<true>(g, T, ph, W, x, y, ye, s);
}

int64_t wq_doubles(const LevelGeom& g) { return (int64_t)g.N * g.ncells() * 6 * g.nt * (g.k + 3) * (g.k + 3); }

void launch_wq(const LevelGeom& g, const FeTables& T, const double* W, double* Wq, cudaStream_t s) {
  if (g.k == 1 && g.q == 0) run_wq<1, 0>(g, T, W, Wq, s);
  else if (g.k == 1 && g.q == 1) run_wq<1, 1>(g, T, W, Wq, s);
  else if (g.k == 2 && g.q == 0) run_wq<2, 0>(g, T, W, Wq, s);
  else if (g.k == 2 && g.q == 1) run_wq<2, 1>(g, T, W, Wq, s);
  else if (g.k == 1 && g.q == 2) run_wq<1, 2>(g, T, W, Wq, s);
  else if (g.k == 1 && g.q == 3) run_wq<1, 3>(g, T, W, Wq, s);
  else if (g.k == 2 && g.q == 2) run_wq<2, 2>(g, T, W, Wq, s);
  else if (g.k == 2 && g.q == 3) run_wq<2, 3>(g, T, W, Wq, s);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

void launch_jacobian_wq(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* Wq,
                        const double* x, double* y, double* ye, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (g.k == 1 && g.q == 0) run_jac<1, 0>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 1 && g.q == 1) run_jac<1, 1>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 2 && g.q == 0) run_jac<2, 0>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 2 && g.q == 1) run_jac<2, 1>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 1 && g.q == 2) run_jac<1, 2>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 1 && g.q == 3) run_jac<1, 3>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 2 && g.q == 2) run_jac<2, 2>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else if (g.k == 2 && g.q == 3) run_jac<2, 3>(g, T, ph, Wq, x, y, ye, s, ev0, ev1);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

// FP64 operations of one (cell, slab) of jac_kernel's sum-factorised algorithm (a
// multiply-add counts 2): interpolation of x (values and both derivatives), x^-
// (values) and the pressure; the pointwise weak form; the test-function contractions.
double jac_flops_per_cell_slab(int k, int q) {
  const double nt = q + 1, nvl = k + 2, npl = k + 1, nq = k + 3, nq2 = nq * nq, nf = 2 * nt;
  const double interp = nf * nvl * nq * 2 * nvl + 2 * nvl * nq * nvl + nt * npl * nq * npl +  // x passes
                        nf * nq2 * 3 * nvl + 2 * nq2 * nvl + nt * nq2 * npl;                // y passes
  const double point = nq2 * (nt + nt * nt * 2 * 4 + nt * (2 * nt + 2 * (1 + nt + nt * nt + 2 * nt)));
  const double test = nf * nvl * nq * 3 * nq + nt * npl * nq * nq + nf * nvl * nvl * 2 * nq + nt * npl * npl * nq;
  return 2.0 * (interp + point + test);
}

void launch_jacobian_f32(const LevelGeom& g, const FeTables& T, const PhysParams& ph, const double* W, const double* x,
                         double* y, double* ye, cudaStream_t s) {
  if (g.k == 1 && g.q == 0) run_element_f32<1, 0>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 1 && g.q == 1) run_element_f32<1, 1>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 2 && g.q == 0) run_element_f32<2, 0>(g, T, ph, W, x, y, ye, s);
  else if (g.k == 2 && g.q == 1) run_element_f32<2, 1>(g, T, ph, W, x, y, ye, s);
  else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
}

void launch_boundary_values(const LevelGeom& g, const FeTables& T, const PhysParams& ph, double* U, cudaStream_t s) {
  const int threads = 256;
  boundary_kernel<<<(unsigned)((g.ndofs + threads - 1) / threads), threads, 0, s>>>(g, T, ph, U);
  WR_LAUNCH_CHECK();
}

void launch_conv_elements(const LevelGeom& g, const FeTables& T, const double* W, void* Ce, int precision,
                          cudaStream_t s) {
  if (precision == WR_FP64) {
    double* c = static_cast<double*>(Ce);
    if (g.k == 1 && g.q == 0) run_conv<1, 0>(g, T, W, c, s);
    else if (g.k == 1 && g.q == 1) run_conv<1, 1>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 0) run_conv<2, 0>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 1) run_conv<2, 1>(g, T, W, c, s);
    else if (g.k == 1 && g.q == 2) run_conv<1, 2>(g, T, W, c, s);
    else if (g.k == 1 && g.q == 3) run_conv<1, 3>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 2) run_conv<2, 2>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 3) run_conv<2, 3>(g, T, W, c, s);
    else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
  } else {
    float* c = static_cast<float*>(Ce);
    if (g.k == 1 && g.q == 0) run_conv<1, 0>(g, T, W, c, s);
    else if (g.k == 1 && g.q == 1) run_conv<1, 1>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 0) run_conv<2, 0>(g, T, W, c, s);
    else if (g.k == 2 && g.q == 1) run_conv<2, 1>(g, T, W, c, s);
    else throw WrError(WR_ERR_ARG, "unsupported (k, q)");
  }
}

void launch_inject(const LevelGeom& gf, const LevelGeom& gc, const double* Wf, double* Wc, cudaStream_t s) {
  const int threads = 256;
  inject_kernel<<<(unsigned)((gc.ndofs + threads - 1) / threads), threads, 0, s>>>(gf, gc, Wf, Wc);
  WR_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- J(W) x without device allocation
// Some callers cannot call cudaMalloc: an application that owns every byte of
// device memory through its own pool, or a latency-critical loop that must not
// pay for the allocator's implicit device synchronisation and its failure modes.
// wr_apply_jacobian_static serves them: it needs no context, and its only
// scratch (the per-element contributions that the assembly kernel sums) lives
// in the fixed file-scope array below, which every GPU that loads this library
// holds until the process exits.
static constexpr int64_t kStaticScratchDoubles = 8ll * 1024 * 1024;  // 64 MiB
static __device__ __align__(256) double g_static_elem_scratch[kStaticScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
double* g_static_scratch_ptr[kMaxDevices] = {};
std::mutex g_static_scratch_mutex;

// Device address of the static scratch on the current device (set up once per device).
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_scratch_mutex);
  if (!g_static_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_elem_scratch);
    if (e != cudaSuccess) return e;
    g_static_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_scratch_ptr[dev];
  return cudaSuccess;
}
}  // namespace

namespace {
int static_fail(int code, const std::string& msg) {
  wr_set_context_free_error("wr_apply_jacobian_static: " + msg);
  return code;
}
}  // namespace

extern "C" int wr_apply_jacobian_static(const wr_problem* p, const double* W, const double* x, double* y,
                                        void* cuda_stream) {
  try {
    if (!p || !W || !x || !y) return static_fail(WR_ERR_ARG, "null pointer");
    if (x == y) return static_fail(WR_ERR_ARG, "x and y alias");
    if ((p->k != 1 && p->k != 2) || (p->q != 0 && p->q != 1))
      return static_fail(WR_ERR_ARG, "unsupported (k, q): k must be 1 or 2 and q 0 or 1");
    if (p->n_fine < 1 || p->n_slabs < 1 || !(p->T > 0.0))
      return static_fail(WR_ERR_ARG, "n_fine, n_slabs and T must be positive");
    if (p->kind != WR_TAYLOR_GREEN && p->kind != WR_POLY && p->kind != WR_FOURIER && p->kind != WR_LID)
      return static_fail(WR_ERR_ARG, "kind is not a Navier-Stokes problem (the heat kinds have no J(W) here)");
    const int64_t nvl = p->k + 2, npl = p->k + 1;
    const int64_t elem = (p->q + 1) * (2 * nvl * nvl + npl * npl);
    const int64_t need = (int64_t)p->n_slabs * p->n_fine * p->n_fine * elem;
    if (need > kStaticScratchDoubles)
      return static_fail(WR_ERR_ARG, "problem needs " + std::to_string(need) +
                                         " doubles of scratch, larger than the static array of " +
                                         std::to_string(kStaticScratchDoubles));
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, stream_dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaStreamGetDevice(s, &stream_dev);
    if (e != cudaSuccess) return static_fail(WR_ERR_CUDA, cudaGetErrorString(e));
    if (stream_dev != dev)
      return static_fail(WR_ERR_ARG, "cuda_stream belongs to device " + std::to_string(stream_dev) +
                                         ", not to the current device " + std::to_string(dev));
    double* scratch = nullptr;
    e = static_scratch(&scratch);
    if (e != cudaSuccess) return static_fail(WR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const LevelGeom g = make_geom(p->n_fine, p->k, p->q, p->n_slabs, p->T);
    const FeTables T = build_tables(p->k, p->q);
    PhysParams ph = {};  // the Jacobian reads nu, conv and T only (Dirichlet rows are the identity)
    ph.kind = WR_FOURIER;
    ph.nu = p->nu;
    ph.conv = p->conv;
    ph.T = p->T;
    ph.n_modes = 0;
    dispatch_element<true>(g, T, ph, W, x, y, scratch, s);
    return WR_OK;
  } catch (const WrError& e) {
    return static_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return static_fail(WR_ERR_CUDA, e.what());
  } catch (...) {
    return static_fail(WR_ERR_CUDA, "unknown exception");
  }
}
