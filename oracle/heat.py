"""Heat-equation waveform relaxation (oracle; test infrastructure only).

Def. heat: u_t - nu lap u = 0 on the unit square with natural (homogeneous
Neumann) boundary conditions, discretised by DG(q) in time (Lagrange basis at
the right-Radau points, as for Navier-Stokes) and continuous Q_k on an n x n
quadrilateral mesh (the quad analogue of the paper's P_k triangles):

    sum_b Kt[a,b] M u_{n,b} + dt nu sum_b Wt[a,b] K u_{n,b} - tau_a(0) M u_{n-1}^- = 0,

with u_{-1}^- = the interpolant of u0 (moved to the right-hand side).  M and K
are the global Q_k mass and stiffness matrices, tensor products of 1D ones on
the Cartesian mesh.  Relaxation (Sec. 3): one vertex-star patch per mesh vertex
holding the nodes of the open star of the vertex -- the vertex and the
interiors of the edges and cells touching it, (2k-1)^2 nodes inside the domain
-- at every temporal DoF of a slab, solved over all slabs by forward
substitution (Eq. waveform_patch_solve); patch matrices are principal
submatrices of the assembled space-time operator; additive scatter with w = 1.
The multigrid hierarchy, transfers, Chebyshev(2) V(2,2) cycle and FGMRES are
those of the Navier-Stokes oracle, for one scalar field.  Sec. 5 solves the
linear system with FGMRES-WRMG to a relative or absolute residual of 1e-6.
"""
import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis import TimeMatrices, equispaced_nodes, gauss_legendre, lagrange
from .solver import Options, arnoldi_ritz_max, chebyshev, fgmres, splitmix64_uniform
from .transfer import interpolation_1d


@dataclasses.dataclass
class HeatProblem:
    """nu: diffusion coefficient; T: slab span; u0: 'paper' = sin(pi x) + cos(2 pi y)
    (Sec. 5), 'cos' = cos(pi x) (a Neumann eigenfunction: u = exp(-nu pi^2 t) cos(pi x))."""

    nu: float = 1.0
    T: float = 0.02
    u0: str = "paper"

    def initial(self, x, y):
        if self.u0 == "cos":
            return np.cos(np.pi * x) + 0.0 * y
        return np.sin(np.pi * x) + np.cos(2.0 * np.pi * y)

    def exact(self, x, y, t):
        """The exact solution (both data choices are sums of Neumann eigenfunctions)."""
        if self.u0 == "cos":
            return np.exp(-self.nu * np.pi ** 2 * t) * np.cos(np.pi * x) + 0.0 * y
        # sin(pi x) is not a Neumann eigenfunction: no closed form is used for it
        raise ValueError("no closed form for the paper's initial data")


def element_1d(p):
    """Reference-interval mass and stiffness matrices of degree-p Lagrange elements."""
    xq, wq = gauss_legendre(p + 2)
    V, D = lagrange(equispaced_nodes(p), xq)
    return np.einsum("iq,jq,q->ij", V, V, wq), np.einsum("iq,jq,q->ij", D, D, wq)


def global_1d(n, p):
    """Global 1D mass and stiffness matrices on [0, 1] with n cells of degree p."""
    m, kk = element_1d(p)
    h = 1.0 / n
    size = n * p + 1
    M = np.zeros((size, size))
    K = np.zeros((size, size))
    for c in range(n):
        s = slice(c * p, c * p + p + 1)
        M[s, s] += h * m
        K[s, s] += kk / h
    return M, K


class HeatDiscretisation:
    def __init__(self, n, k, q, N, problem):
        self.n, self.k, self.q, self.N = n, k, q, N
        self.pb = problem
        self.dt = problem.T / N
        self.nv = n * k + 1
        self.S = self.nv ** 2
        self.nt = q + 1
        self.ndofs = N * self.nt * self.S
        self.tm = TimeMatrices(q)
        M1, K1 = global_1d(n, k)
        M1, K1 = sp.csr_matrix(M1), sp.csr_matrix(K1)
        self.M = sp.kron(M1, M1).tocsr()                       # (y, x) ordering
        self.K = (sp.kron(K1, M1) + sp.kron(M1, K1)).tocsr()
        self.initial_state = None

    def block(self, slab, a):
        return (slab * self.nt + a) * self.S

    def node_coords(self):
        return np.linspace(0.0, 1.0, self.nv)

    def initial_values(self):
        """u(0): the given spatial block, else the nodal interpolant of u0."""
        if self.initial_state is not None:
            return self.initial_state.copy()
        x = self.node_coords()
        X, Y = np.meshgrid(x, x, indexing="xy")
        return self.pb.initial(X, Y).ravel()

    def slab_blocks(self):
        tm = self.tm
        D = sp.kron(tm.Kt, self.M) + self.dt * self.pb.nu * sp.kron(tm.Wt, self.K)
        E = np.zeros((self.nt, self.nt))
        E[:, self.nt - 1] = -tm.tau0
        return D.tocsr(), sp.kron(E, self.M).tocsr()

    def jacobian(self):
        D, L = self.slab_blocks()
        blocks = [[None] * self.N for _ in range(self.N)]
        for n in range(self.N):
            blocks[n][n] = D
            if n > 0:
                blocks[n][n - 1] = L
        return sp.bmat(blocks, format="csr")

    def rhs(self):
        """The initial-data term tau_a(0) M u(0) in the rows of slab 0."""
        b = np.zeros(self.ndofs)
        Mu = self.M @ self.initial_values()
        for a in range(self.nt):
            b[self.block(0, a):self.block(0, a) + self.S] = self.tm.tau0[a] * Mu
        return b

    def residual(self, U):
        return self.jacobian() @ U - self.rhs()


def heat_patch_spatial(d, I, J):
    """Nodes of the open star of vertex (I, J), lexicographic (y-major, x fastest)."""
    k, nv = d.k, d.nv
    xs = [g for g in range((I - 1) * k + 1, (I + 1) * k) if 0 <= g < nv]
    ys = [g for g in range((J - 1) * k + 1, (J + 1) * k) if 0 <= g < nv]
    return np.array([gy * nv + gx for gy in ys for gx in xs], dtype=np.int64)


def heat_patch_dofs(d, patch, slab):
    n1 = d.n + 1
    sidx = heat_patch_spatial(d, patch % n1, patch // n1)
    return np.concatenate([d.block(slab, a) + sidx for a in range(d.nt)])


class HeatSmoother:
    """Vertex-star waveform relaxation: sum_i R_i^T A_i^{-1} R_i r, A_i = J[P_i, P_i]
    solved by forward substitution over slabs with dense LU per slab block."""

    def __init__(self, d, J):
        self.d = d
        self.npatch = (d.n + 1) ** 2
        self.idx = [[heat_patch_dofs(d, i, s) for s in range(d.N)] for i in range(self.npatch)]
        self.lu = [[sla.lu_factor(J[ix][:, ix].toarray(), check_finite=False) for ix in row] for row in self.idx]
        self.sub = [[None] + [J[row[s]][:, row[s - 1]].toarray() for s in range(1, d.N)] for row in self.idx]

    def apply(self, r):
        out = np.zeros_like(r)
        for i in range(self.npatch):
            prev = None
            for s in range(self.d.N):
                ix = self.idx[i][s]
                rhs = r[ix].copy()
                if s > 0:
                    rhs -= self.sub[i][s] @ prev
                prev = sla.lu_solve(self.lu[i][s], rhs, check_finite=False)
                np.add.at(out, ix, prev)
        return out


def heat_prolongation(fine, coarse):
    P1 = sp.csr_matrix(interpolation_1d(coarse.n, fine.k))
    return sp.kron(sp.identity(fine.N * fine.nt), sp.kron(P1, P1)).tocsr()


class HeatCoarseSolver:
    """Exact solve on the coarsest level: dense LU per slab block, forward substitution."""

    def __init__(self, d, J):
        self.d = d
        self.idx = [np.arange(d.block(n, 0), d.block(n + 1, 0)) for n in range(d.N)]
        self.lu = [sla.lu_factor(J[ix][:, ix].toarray(), check_finite=False) for ix in self.idx]
        self.sub = [None] + [J[self.idx[n]][:, self.idx[n - 1]].toarray() for n in range(1, d.N)]

    def solve(self, b):
        out = np.zeros_like(b)
        prev = None
        for n in range(self.d.N):
            rhs = b[self.idx[n]].copy()
            if n > 0:
                rhs -= self.sub[n] @ prev
            prev = sla.lu_solve(self.lu[n], rhs, check_finite=False)
            out[self.idx[n]] = prev
        return out


class HeatHierarchy:
    """Levels n_coarse, 2 n_coarse, ..., n_fine; the operator is linear, so every
    level's matrix, smoother and eigen-estimate is set up once."""

    def __init__(self, n_fine, n_coarse, k, q, N, problem, opts=None):
        self.opts = opts or Options()
        ns = []
        n = n_fine
        while n >= n_coarse:
            ns.append(n)
            n //= 2
        self.discs = [HeatDiscretisation(n, k, q, N, problem) for n in ns[::-1]]
        self.J = [d.jacobian() for d in self.discs]
        self.P = [None] + [heat_prolongation(self.discs[l], self.discs[l - 1]) for l in range(1, len(ns))]
        self.coarse = HeatCoarseSolver(self.discs[0], self.J[0])
        self.smoothers = [None] + [HeatSmoother(self.discs[l], self.J[l]) for l in range(1, len(ns))]
        self.lam = [None]
        for l in range(1, len(ns)):
            J, M = self.J[l], self.smoothers[l]
            v0 = splitmix64_uniform(l, self.discs[l].ndofs)
            self.lam.append(arnoldi_ritz_max(lambda v: M.apply(J @ v), v0, self.opts.eig_steps))

    @property
    def fine(self):
        return self.discs[-1]

    def vcycle(self, b):
        L = len(self.discs) - 1
        bs, xs = [None] * (L + 1), [None] * (L + 1)
        bs[L] = b
        for l in range(L, 0, -1):
            Jop = lambda v, J=self.J[l]: J @ v
            xs[l] = chebyshev(Jop, self.smoothers[l].apply, bs[l], None, self.lam[l], self.opts)
            bs[l - 1] = self.P[l].T @ (bs[l] - self.J[l] @ xs[l])
        xs[0] = self.coarse.solve(bs[0])
        for l in range(1, L + 1):
            Jop = lambda v, J=self.J[l]: J @ v
            xs[l] = chebyshev(Jop, self.smoothers[l].apply, bs[l], xs[l] + self.P[l] @ xs[l - 1],
                              self.lam[l], self.opts)
        return xs[L]


def heat_solve(hier, rtol=1e-6, atol=1e-6, restart=30, maxit=200):
    """Sec. 5: FGMRES preconditioned by one V(2,2) WRMG cycle, from a zero guess, to
    ||r|| <= max(rtol ||b||, atol).  Returns (U, FGMRES iterations)."""
    b = hier.fine.rhs()
    J = hier.J[-1]
    return fgmres(lambda v: J @ v, hier.vcycle, b, max(rtol * np.linalg.norm(b), atol), restart, maxit)
