// Host construction of the reference-element and DG(q) time tables.
//
// Space: Lagrange Q_p on p+1 equispaced nodes of [0, 1] (velocity p = k+1,
// pressure p = k, Taylor-Hood, Def. "Navier-Stokes equations").  Gauss-Legendre
// points are found by Newton's method on the Legendre polynomial P_nq (three-
// term recurrence), right-Radau points (Radau IIA abscissae) by Newton's method
// on P_{q+1}(2s-1) - P_q(2s-1).  Time: DG(q) of Eq. dgintime with a Lagrange
// basis at the right-Radau points.
#include <cmath>

#include "wrmg_internal.h"

namespace {

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2 * j - 1) * x * p1 - (j - 1) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss-Legendre points/weights on [0, 1].
void gauss01(int nq, double* x, double* w) {
  for (int i = 0; i < nq; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (nq + 0.5));  // initial guess (descending)
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(nq, t, &p, &dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p, dp;
    legendre(nq, t, &p, &dp);
    int j = nq - 1 - i;  // ascending order
    x[j] = 0.5 * (t + 1.0);
    w[j] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) mapped by 1/2
  }
}

// Right-Radau points on [0, 1]: zeros of P_s(y) - P_{s-1}(y), y = 2s-1; y = 1 is one of them.
void radau01(int q, double* s) {
  int ns = q + 1;
  s[ns - 1] = 1.0;
  if (ns == 1) return;
  // remaining ns-1 zeros lie in (-1, 1): deflate the known root y = 1
  for (int i = 0; i < ns - 1; ++i) {
    double y = -std::cos(M_PI * (2 * i + 1) / (2 * ns - 1));
    for (int it = 0; it < 200; ++it) {
      double pa, dpa, pb, dpb;
      legendre(ns, y, &pa, &dpa);
      legendre(ns - 1, y, &pb, &dpb);
      double f = (pa - pb) / (y - 1.0);
      double df = ((dpa - dpb) - f) / (y - 1.0);
      double d = f / df;
      y -= d;
      if (std::fabs(d) < 1e-16) break;
    }
    s[i] = 0.5 * (y + 1.0);
  }
  for (int i = 0; i < ns - 1; ++i)
    for (int j = i + 1; j < ns - 1; ++j)
      if (s[j] < s[i]) std::swap(s[i], s[j]);
}

// Lagrange basis l_i and l_i' on the given nodes at x.
void lagr(int np, const double* nodes, double x, double* v, double* d) {
  for (int i = 0; i < np; ++i) {
    double prod = 1.0, der = 0.0;
    for (int m = 0; m < np; ++m) {
      if (m == i) continue;
      double term = 1.0 / (nodes[i] - nodes[m]);
      for (int j = 0; j < np; ++j)
        if (j != i && j != m) term *= (x - nodes[j]) / (nodes[i] - nodes[j]);
      der += term;
      prod *= (x - nodes[m]) / (nodes[i] - nodes[m]);
    }
    v[i] = prod;
    if (d) d[i] = der;
  }
}

}  // namespace

FeTables build_tables(int k, int q) {
  FeTables T = {};
  const int nq = k + 3, nvl = k + 2, npl = k + 1, nt = q + 1;
  gauss01(nq, T.xq, T.wq);
  double vnodes[WR_MAX_NVL], pnodes[WR_MAX_NPL];
  for (int i = 0; i < nvl; ++i) vnodes[i] = double(i) / (nvl - 1);
  for (int i = 0; i < npl; ++i) pnodes[i] = npl == 1 ? 0.0 : double(i) / (npl - 1);
  for (int g = 0; g < nq; ++g) {
    lagr(nvl, vnodes, T.xq[g], T.Bv[g], T.Dv[g]);
    lagr(npl, pnodes, T.xq[g], T.Bp[g], nullptr);
  }
  for (int i = 0; i < nvl; ++i)
    for (int j = 0; j < nvl; ++j)
      for (int g = 0; g < nq; ++g) {
        T.m1[i][j] += T.wq[g] * T.Bv[g][i] * T.Bv[g][j];
        T.k1[i][j] += T.wq[g] * T.Dv[g][i] * T.Dv[g][j];
      }
  for (int p = 0; p < npl; ++p) {
    for (int g = 0; g < nq; ++g) T.mp1[p] += T.wq[g] * T.Bp[g][p];
    for (int v = 0; v < nvl; ++v)
      for (int g = 0; g < nq; ++g) {
        T.d1[p][v] += T.wq[g] * T.Bp[g][p] * T.Dv[g][v];
        T.c1[p][v] += T.wq[g] * T.Bp[g][p] * T.Bv[g][v];
      }
  }
  // time
  radau01(q, T.tnode);
  double tx[WR_MAX_NT + 2], tw[WR_MAX_NT + 2];
  const int ntg = q + 3;  // exact for the degree-3q integrands below
  gauss01(ntg, tx, tw);
  double v0[WR_MAX_NT];
  lagr(nt, T.tnode, 0.0, v0, nullptr);
  for (int a = 0; a < nt; ++a) T.tau0[a] = v0[a];
  for (int g = 0; g < ntg; ++g) {
    double v[WR_MAX_NT], d[WR_MAX_NT];
    lagr(nt, T.tnode, tx[g], v, d);
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) {
        T.Kt[a][b] += tw[g] * v[a] * d[b];
        T.Wt[a][b] += tw[g] * v[a] * v[b];
        for (int c = 0; c < nt; ++c) T.T3[a][b][c] += tw[g] * v[a] * v[b] * v[c];
      }
  }
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) T.Kt[a][b] += T.tau0[a] * T.tau0[b];
  gauss01(q + 2, T.tq, T.wtq);
  for (int g = 0; g < q + 2; ++g) {
    double v[WR_MAX_NT];
    lagr(nt, T.tnode, T.tq[g], v, nullptr);
    for (int a = 0; a < nt; ++a) T.Tq[a][g] = v[a];
  }
  // prolongation weights: fine node r of a coarse cell sits at xi = r / (2p)
  for (int r = 0; r <= 2 * (nvl - 1); ++r) lagr(nvl, vnodes, r / (2.0 * (nvl - 1)), T.pv[r], nullptr);
  for (int r = 0; r <= 2 * (npl - 1); ++r) {
    if (npl == 1) { T.pp[r][0] = 1.0; continue; }
    lagr(npl, pnodes, r / (2.0 * (npl - 1)), T.pp[r], nullptr);
  }
  // exact zeros where nodes coincide (nested equispaced nodes)
  for (auto& row : T.pv)
    for (double& x : row)
      if (std::fabs(x) < 1e-15) x = 0.0;
  for (auto& row : T.pp)
    for (double& x : row)
      if (std::fabs(x) < 1e-15) x = 0.0;
  return T;
}
