"""1D building blocks of the discretisation (oracle; test infrastructure only).

Space: continuous Lagrange Q_p on equispaced nodes of the reference interval
[0, 1]; velocity uses p = k+1, pressure p = k (Taylor-Hood, Def. "Navier-Stokes
equations").  Time: discontinuous Galerkin DG(q) (Def. "Temporal
discretisation", Eq. dgintime) with a Lagrange basis at the q+1 right-Radau
(Radau IIA) points of each slab, so the last temporal degree of freedom is the
value at the slab end t_{n+1}^- that the upwind jump term reads.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def equispaced_nodes(p):
    """The p+1 equispaced Lagrange nodes of Q_p on [0, 1]."""
    return np.linspace(0.0, 1.0, p + 1)


def lagrange(nodes, x):
    """Values and first derivatives of the Lagrange basis on ``nodes`` at ``x``.

    Returns (V, D) with V[i, j] = l_i(x_j) and D[i, j] = l_i'(x_j), written out
    from the product formula l_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = len(nodes)
    V = np.ones((p, len(x)))
    D = np.zeros((p, len(x)))
    for i in range(p):
        for m in range(p):
            if m == i:
                continue
            V[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for m in range(p):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(p):
                if j == i or j == m:
                    continue
                term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            D[i] += term
    return V, D


def gauss_legendre(nq):
    """nq-point Gauss-Legendre rule mapped to [0, 1] (exact to degree 2nq-1)."""
    x, w = npleg.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def radau_right_nodes(q):
    """The q+1 right-Radau points on [0, 1] (Radau IIA abscissae).

    They are the zeros of P_{q+1}(2s-1) - P_q(2s-1); the last one is s = 1.
    """
    s = q + 1
    cp = np.zeros(s + 1)
    cp[s] = 1.0
    cm = np.zeros(s + 1)
    cm[s - 1] = 1.0
    roots = npleg.legroots(cp - cm)
    nodes = np.sort(0.5 * (np.real(roots) + 1.0))
    nodes[-1] = 1.0
    return nodes


class TimeMatrices:
    """Slab-local DG(q) matrices on the reference slab s in [0, 1], t = t_n + s dt.

    With U(s) = sum_b tau_b(s) U_b on slab n and test function tau_a(s):

    * ``Kt[a, b] = int tau_a tau_b' ds + tau_a(0) tau_b(0)`` -- the time
      derivative plus the part of the upwind jump [[U_n]] psi_n^+ that falls
      on slab n (Eq. dgintime);
    * ``tau0[a] = tau_a(0)`` -- the jump's coupling to the previous slab's end
      value U_n^- (the last temporal DoF of slab n-1, or the initial data);
    * ``Wt[a, b] = int tau_a tau_b ds`` -- the time mass (multiplies dt);
    * ``T3[a, b, c] = int tau_a tau_b tau_c ds`` -- the time tensor of the
      quadratic convection term (multiplies dt);
    * ``tq, wq, Tq`` -- the (q+2)-point Gauss rule in time used for the
      forcing, and Tq[a, g] = tau_a(tq_g).
    """

    def __init__(self, q):
        self.q = q
        self.nodes = radau_right_nodes(q)
        nq = q + 3  # exact for the degree-3q products below (q <= 3)
        xs, ws = gauss_legendre(nq)
        V, D = lagrange(self.nodes, xs)
        V0, _ = lagrange(self.nodes, [0.0])
        self.tau0 = V0[:, 0].copy()
        self.Kt = np.einsum("ag,bg,g->ab", V, D, ws) + np.outer(self.tau0, self.tau0)
        self.Wt = np.einsum("ag,bg,g->ab", V, V, ws)
        self.T3 = np.einsum("ag,bg,cg,g->abc", V, V, V, ws)
        self.tq, self.wq = gauss_legendre(q + 2)
        self.Tq, _ = lagrange(self.nodes, self.tq)
