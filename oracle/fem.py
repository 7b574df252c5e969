"""Space-time Taylor-Hood discretisation of Navier-Stokes (oracle; test
infrastructure only).

Follows Eq. nsfem with the viscosity/convection scaling
    u_t + conv (u.grad)u + grad p - nu lap u = f,   div u = 0
(the paper's form is conv = R, nu = 1; the two agree under t -> nu t), on a
uniform n x n quadrilateral mesh of the unit square with Q_{k+1}^2 / Q_k
Taylor-Hood elements (the quadrilateral analogue of the paper's P_{k+1}/P_k)
and DG(q) in time (Def. "Temporal discretisation").

Weak form, slab n, test psi = tau_a(s) phi_i (velocity), tau_a chi_i (pressure):

  F_u = sum_b Kt[a,b] (U_b, phi) - tau_a(0) (U_n^-, phi)
        + dt [ conv sum_{b,c} T3[a,b,c] ((U_b.grad) U_c, phi)
               + sum_b Wt[a,b] (Phi_b, div phi) + nu sum_b Wt[a,b] (grad U_b, grad phi)
               - int_0^1 tau_a (f, phi) ds ]
  F_p = dt sum_b Wt[a,b] (div U_b, chi)

Signs are those printed in Eq. nsfem: +(Phi, div psi) and +(div U, chi), so the
discrete Phi approximates minus the strong-form pressure p.  U_0^- is the nodal
interpolant of u(0) (the "weakly imposed" initial condition of the Chorin
problem); Dirichlet velocity data are the nodal interpolant of the boundary
values at every temporal node (strong), and those rows read U - g.

Quadrature: (k+3)-point Gauss-Legendre per space direction (exact for every
polynomial integrand here) and the (q+2)-point Gauss rule in time for f.

Canonical global index (the bit-exact contract with the CUDA path):
    ((slab*(q+1) + a) * S + field_offset + y*nf + x),
with S = 2 nv^2 + np^2, fields u_x, u_y, p in that order, nv = n(k+1)+1,
np = nk+1 nodes per direction, x fastest.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .basis import TimeMatrices, equispaced_nodes, gauss_legendre, lagrange


@dataclass
class Problem:
    """What is solved: the PDE parameters and the data.

    kind: 'taylor_green' -- decaying Taylor-Green (Chorin) vortex, f = 0,
              u = (-cos(pi x) sin(pi y), sin(pi x) cos(pi y)) exp(-2 nu pi^2 t),
              p = -(cos(2 pi x) + cos(2 pi y)) exp(-4 nu pi^2 t) / 4 (conv = 1);
          'poly'  -- u = (y^2, x^2)(1+t), p = x + y - 1 (q >= 1), or the
              time-constant u = (y^2, x^2) when ``steady`` (any q); it lies in
              the discrete space for k >= 1, so the discrete solution is exact;
          'fourier' -- no-slip walls, u(0) = 0, time-independent divergence-free
              forcing f = sum_j amp_j (d_y psi_j, -d_x psi_j),
              psi_j = sin(mx_j pi x) sin(my_j pi y);
          'lid' -- lid-driven cavity (Sec. 4): u = (1, 0) on the open top edge
              y = 1, 0 < x < 1, zero on the other walls and at the two top
              corners, u(0) = 0, f = 0 (no exact solution).
    """

    kind: str = "taylor_green"
    nu: float = 1e-2
    conv: float = 1.0
    T: float = 1.0
    t0: float = 0.0          # time at the start of slab 0: the slabs cover [t0, t0 + T]
    steady: bool = False
    mx: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    my: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    amp: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def exact_velocity(self, x, y, t):
        if self.kind == "taylor_green":
            e = np.exp(-2.0 * self.nu * np.pi ** 2 * t)
            return (-np.cos(np.pi * x) * np.sin(np.pi * y) * e,
                    np.sin(np.pi * x) * np.cos(np.pi * y) * e)
        if self.kind == "poly":
            s = 1.0 if self.steady else 1.0 + t
            return y * y * s, x * x * s
        return 0.0 * x, 0.0 * y

    def boundary_velocity(self, x, y, t):
        """The Dirichlet data on the boundary nodes (x, y at the nodes)."""
        if self.kind == "lid":
            lid = (y == 1.0) & (x > 0.0) & (x < 1.0)
            return np.where(lid, 1.0, 0.0) + 0.0 * x, 0.0 * x
        return self.exact_velocity(x, y, t)

    def exact_pressure(self, x, y, t):
        """Strong-form pressure p (the discrete Phi approximates -p)."""
        if self.kind == "taylor_green":
            return -0.25 * (np.cos(2 * np.pi * x) + np.cos(2 * np.pi * y)) * np.exp(
                -4.0 * self.nu * np.pi ** 2 * t)
        if self.kind == "poly":
            return x + y - 1.0
        return 0.0 * x

    def forcing(self, x, y, t):
        if self.kind == "taylor_green":
            return 0.0 * x, 0.0 * y
        if self.kind == "poly":
            nu, c = self.nu, self.conv
            if self.steady:
                return (2 * c * x * x * y + 1.0 - 2 * nu + 0.0 * t,
                        2 * c * x * y * y + 1.0 - 2 * nu + 0.0 * t)
            s = 1.0 + t
            return (y * y + 2 * c * x * x * y * s * s + 1.0 - 2 * nu * s,
                    x * x + 2 * c * x * y * y * s * s + 1.0 - 2 * nu * s)
        fx = 0.0 * x
        fy = 0.0 * y
        for m, n, a in zip(self.mx, self.my, self.amp):
            fx = fx + a * n * np.pi * np.sin(m * np.pi * x) * np.cos(n * np.pi * y)
            fy = fy - a * m * np.pi * np.cos(m * np.pi * x) * np.sin(n * np.pi * y)
        return fx + 0.0 * t, fy + 0.0 * t


class Discretisation:
    """One level of the space-time discretisation: mesh n x n, Q_{k+1}^2/Q_k, DG(q), N slabs."""

    def __init__(self, n, k, q, N, problem):
        self.n, self.k, self.q, self.N = n, k, q, N
        self.pb = problem
        self.h = 1.0 / n
        self.dt = problem.T / N
        self.nv = n * (k + 1) + 1
        self.np_ = n * k + 1
        self.S = 2 * self.nv ** 2 + self.np_ ** 2
        self.nt = q + 1
        self.ndofs = N * self.nt * self.S
        self.off_p = 2 * self.nv ** 2
        self.tm = TimeMatrices(q)
        # u(t0) for the jump of slab 0: the exact data unless a spatial block is set here
        self.initial_state = None
        self._tables()
        self._linear_matrices()

    # ------------------------------------------------------------ indexing
    def vel_index(self, c, gx, gy):
        return c * self.nv ** 2 + gy * self.nv + gx

    def pres_index(self, px, py):
        return self.off_p + py * self.np_ + px

    def block(self, slab, a):
        """Offset of temporal DoF a of ``slab`` in the global vector."""
        return (slab * self.nt + a) * self.S

    def spatial_dirichlet(self):
        """Boolean mask over one spatial block: velocity nodes on the boundary."""
        m = np.zeros(self.S, dtype=bool)
        nv = self.nv
        g = np.arange(nv)
        edge = np.zeros((nv, nv), dtype=bool)
        edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
        for c in range(2):
            m[c * nv * nv:(c + 1) * nv * nv] = edge.ravel()
        del g
        return m

    def dirichlet_mask(self):
        return np.tile(self.spatial_dirichlet(), self.N * self.nt)

    def node_coords(self):
        """Physical coordinates of velocity and pressure nodes (1D arrays)."""
        return (np.linspace(0, 1, self.nv), np.linspace(0, 1, self.np_))

    def time_nodes(self, slab):
        return self.pb.t0 + (slab + self.tm.nodes) * self.dt

    # ------------------------------------------------------------ element tables
    def _tables(self):
        k = self.k
        self.nq = k + 3
        xq, wq = gauss_legendre(self.nq)
        self.xq1, self.wq1 = xq, wq
        vv, dv = lagrange(equispaced_nodes(k + 1), xq)      # (k+2, nq)
        vp, _ = lagrange(equispaced_nodes(k), xq)           # (k+1, nq)
        nq = self.nq
        # 2D tables, local node (j, i) -> j*(p+1)+i, point (qy, qx) -> qy*nq+qx
        self.Vv = np.einsum("jy,ix->jiyx", vv, vv).reshape((k + 2) ** 2, nq * nq)
        self.Dxv = np.einsum("jy,ix->jiyx", vv, dv).reshape((k + 2) ** 2, nq * nq) / self.h
        self.Dyv = np.einsum("jy,ix->jiyx", dv, vv).reshape((k + 2) ** 2, nq * nq) / self.h
        self.Vp = np.einsum("jy,ix->jiyx", vp, vp).reshape((k + 1) ** 2, nq * nq)
        self.wq2 = np.einsum("y,x->yx", wq, wq).ravel() * self.h * self.h
        n = self.n
        I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        I, J = I.ravel(), J.ravel()                          # cell (I, J), cell id J*n+I
        self.cellI, self.cellJ = I, J
        li = np.arange(k + 2)
        gx = I[:, None, None] * (k + 1) + li[None, None, :]
        gy = J[:, None, None] * (k + 1) + li[None, :, None]
        self.cell_vnodes = (gy * self.nv + gx).reshape(n * n, (k + 2) ** 2)
        lp = np.arange(k + 1)
        px = I[:, None, None] * k + lp[None, None, :]
        py = J[:, None, None] * k + lp[None, :, None]
        self.cell_pnodes = (py * self.np_ + px).reshape(n * n, (k + 1) ** 2)
        # physical quadrature points per cell
        qx = np.tile(xq, nq)
        qy = np.repeat(xq, nq)
        self.qpx = (I[:, None] + qx[None, :]) * self.h
        self.qpy = (J[:, None] + qy[None, :]) * self.h

    def _assemble(self, rows_local, cols_local, vals, shape):
        """COO assembly of per-cell blocks: rows/cols (ncell, a), (ncell, b); vals (ncell, a, b)."""
        r = np.broadcast_to(rows_local[:, :, None], vals.shape).ravel()
        c = np.broadcast_to(cols_local[:, None, :], vals.shape).ravel()
        return sp.coo_matrix((vals.ravel(), (r, c)), shape=shape).tocsr()

    def _linear_matrices(self):
        """Spatial S x S matrices of the whole mesh: velocity mass Mv, velocity
        stiffness Kv and the symmetric pressure coupling G (rows of velocity tests
        against pressure trials: (chi_j, d_c phi_i); rows of pressure tests: its
        transpose)."""
        self.Mv, self.Kv, self.G = self.linear_matrices_on(np.arange(self.n * self.n))
        w = self.wq2
        nc = self.n * self.n
        Mp = self._assemble(self.cell_pnodes, self.cell_pnodes,
                            np.broadcast_to(np.einsum("iq,jq,q->ij", self.Vp, self.Vp, w),
                                            (nc, (self.k + 1) ** 2, (self.k + 1) ** 2)),
                            (self.np_ ** 2, self.np_ ** 2))
        self.pressure_weights = np.asarray(Mp.sum(axis=1)).ravel()   # int chi_j

    def linear_matrices_on(self, cells):
        """(Mv, Kv, G) assembled over the cells with ids in ``cells`` only."""
        S, nv2 = self.S, self.nv ** 2
        w = self.wq2
        Me = np.einsum("iq,jq,q->ij", self.Vv, self.Vv, w)
        Ke = np.einsum("iq,jq,q->ij", self.Dxv, self.Dxv, w) + np.einsum(
            "iq,jq,q->ij", self.Dyv, self.Dyv, w)
        Gx = np.einsum("iq,jq,q->ij", self.Dxv, self.Vp, w)   # (vel i, pres j)
        Gy = np.einsum("iq,jq,q->ij", self.Dyv, self.Vp, w)
        cells = np.asarray(cells, dtype=np.int64)
        nc = len(cells)
        blocks_M, blocks_K, blocks_G = [], [], []
        for c in range(2):
            rv = self.cell_vnodes[cells] + c * nv2
            blocks_M.append(self._assemble(rv, rv, np.broadcast_to(Me, (nc,) + Me.shape), (S, S)))
            blocks_K.append(self._assemble(rv, rv, np.broadcast_to(Ke, (nc,) + Ke.shape), (S, S)))
            Ge = Gx if c == 0 else Gy
            rp = self.cell_pnodes[cells] + self.off_p
            blocks_G.append(self._assemble(rv, rp, np.broadcast_to(Ge, (nc,) + Ge.shape), (S, S)))
        G = blocks_G[0] + blocks_G[1]
        return blocks_M[0] + blocks_M[1], blocks_K[0] + blocks_K[1], (G + G.T).tocsr()

    # ------------------------------------------------------------ fields at quadrature points
    def _vel_at_q(self, uc):
        """uc: spatial vector of one velocity component (nv^2). Returns value, d/dx, d/dy
        at the quadrature points of every cell, each (ncell, nq^2)."""
        loc = uc[self.cell_vnodes]
        return loc @ self.Vv, loc @ self.Dxv, loc @ self.Dyv

    def convection_matrix(self, w, cells=None):
        """Spatial S x S matrix of the linearised convection about the spatial
        velocity field w (a spatial block): rows (c, i), cols (d, j),
        int phi_i [ delta_cd (w.grad) phi_j + phi_j d_d w_c ]; over every cell, or
        over the cells with ids in ``cells`` only."""
        S, nv2 = self.S, self.nv ** 2
        cells = np.arange(self.n * self.n) if cells is None else np.asarray(cells, dtype=np.int64)
        wx, wxx, wxy = (f[cells] for f in self._vel_at_q(w[:nv2]))
        wy, wyx, wyy = (f[cells] for f in self._vel_at_q(w[nv2:2 * nv2]))
        W = self.wq2
        adv = wx[:, None, :] * self.Dxv[None] + wy[:, None, :] * self.Dyv[None]   # (cell, j, q)
        base = np.einsum("iq,cjq,q->cij", self.Vv, adv, W)
        mass_w = lambda g: np.einsum("iq,jq,cq,q->cij", self.Vv, self.Vv, g, W)
        grads = [[wxx, wxy], [wyx, wyy]]   # grads[c][d] = d_d w_c
        out = None
        for c in range(2):
            for d in range(2):
                vals = mass_w(grads[c][d])
                if c == d:
                    vals = vals + base
                A = self._assemble(self.cell_vnodes[cells] + c * nv2, self.cell_vnodes[cells] + d * nv2, vals,
                                   (S, S))
                out = A if out is None else out + A
        return out

    # ------------------------------------------------------------ data
    def boundary_values(self):
        """Global vector holding g at Dirichlet velocity DoFs (zero elsewhere)."""
        xv, _ = self.node_coords()
        X, Y = np.meshgrid(xv, xv, indexing="xy")
        mask = self.spatial_dirichlet()
        g = np.zeros(self.ndofs)
        nv2 = self.nv ** 2
        for n in range(self.N):
            for a, t in enumerate(self.time_nodes(n)):
                ux, uy = self.pb.boundary_velocity(X, Y, t)
                blk = np.zeros(self.S)
                blk[:nv2] = np.broadcast_to(ux, X.shape).ravel()
                blk[nv2:2 * nv2] = np.broadcast_to(uy, X.shape).ravel()
                off = self.block(n, a)
                g[off:off + self.S] = np.where(mask, blk, 0.0)
        return g

    def initial_velocity(self):
        """Spatial block holding u(t0) (pressure part zero): the velocity part of
        ``initial_state`` when it is set (e.g. the end state of a previous time
        step), else the nodal interpolant of the exact u(t0)."""
        nv2 = self.nv ** 2
        if self.initial_state is not None:
            u0 = np.zeros(self.S)
            u0[:2 * nv2] = self.initial_state[:2 * nv2]
            return u0
        xv, _ = self.node_coords()
        X, Y = np.meshgrid(xv, xv, indexing="xy")
        ux, uy = self.pb.exact_velocity(X, Y, self.pb.t0)
        u0 = np.zeros(self.S)
        nv2 = self.nv ** 2
        u0[:nv2] = np.broadcast_to(ux, X.shape).ravel()
        u0[nv2:2 * nv2] = np.broadcast_to(uy, X.shape).ravel()
        return u0

    def interpolant(self):
        """Global nodal interpolant of the exact (u, Phi = -p) at every temporal node."""
        xv, xp = self.node_coords()
        X, Y = np.meshgrid(xv, xv, indexing="xy")
        XP, YP = np.meshgrid(xp, xp, indexing="xy")
        U = np.zeros(self.ndofs)
        nv2 = self.nv ** 2
        for n in range(self.N):
            for a, t in enumerate(self.time_nodes(n)):
                ux, uy = self.pb.exact_velocity(X, Y, t)
                p = self.pb.exact_pressure(XP, YP, t)
                off = self.block(n, a)
                U[off:off + nv2] = np.broadcast_to(ux, X.shape).ravel()
                U[off + nv2:off + 2 * nv2] = np.broadcast_to(uy, X.shape).ravel()
                U[off + self.off_p:off + self.S] = -np.broadcast_to(p, XP.shape).ravel()
        return U

    def forcing_vector(self, slab):
        """int_{I_n} tau_a (f, phi_i) dt for every a: array (q+1, S) (velocity rows)."""
        tm = self.tm
        out = np.zeros((self.nt, self.S))
        nv2 = self.nv ** 2
        for g, (sg, wg) in enumerate(zip(tm.tq, tm.wq)):
            t = self.pb.t0 + (slab + sg) * self.dt
            fx, fy = self.pb.forcing(self.qpx, self.qpy, t)
            fx = np.broadcast_to(fx, self.qpx.shape)
            fy = np.broadcast_to(fy, self.qpy.shape)
            for c, fc in enumerate((fx, fy)):
                loc = np.einsum("cq,iq,q->ci", fc, self.Vv, self.wq2)     # (cell, i)
                vec = np.zeros(nv2)
                np.add.at(vec, self.cell_vnodes.ravel(), loc.ravel())
                for a in range(self.nt):
                    out[a, c * nv2:(c + 1) * nv2] += self.dt * wg * tm.Tq[a, g] * vec
        return out

    # ------------------------------------------------------------ residual and Jacobian
    def _slab(self, U, slab):
        return U[self.block(slab, 0):self.block(slab + 1, 0)].reshape(self.nt, self.S)

    def residual(self, U):
        """Nonlinear space-time residual F(U) of Eq. nsfem (Dirichlet rows: U - g)."""
        F = np.zeros(self.ndofs)
        for n in range(self.N):
            F[self.block(n, 0):self.block(n + 1, 0)] = self.residual_slab(U, n)
        return F

    def residual_slab(self, U, n):
        """The rows of F(U) that belong to slab n (they read slabs n and n-1 of U)."""
        tm, dt, nu, cv = self.tm, self.dt, self.pb.nu, self.pb.conv
        nv2 = self.nv ** 2
        if n == 0:
            u_prev = self.initial_velocity()
        else:
            u_prev = self._slab(U, n - 1)[self.nt - 1].copy()
            u_prev[self.off_p:] = 0.0
        Un = self._slab(U, n)
        # velocity values/gradients at quadrature points for each temporal DoF
        fields = [[self._vel_at_q(Un[b, c * nv2:(c + 1) * nv2]) for c in range(2)]
                  for b in range(self.nt)]
        Fn = np.zeros((self.nt, self.S))
        for a in range(self.nt):
            r = np.zeros(self.S)
            for b in range(self.nt):
                r += tm.Kt[a, b] * (self.Mv @ Un[b])
                r += dt * tm.Wt[a, b] * (nu * (self.Kv @ Un[b]) + self.G @ Un[b])
            r -= tm.tau0[a] * (self.Mv @ u_prev)
            for c in range(2):
                integrand = np.zeros_like(self.qpx)
                for b in range(self.nt):
                    for e in range(self.nt):
                        ub = fields[b]
                        ue = fields[e][c]
                        integrand += tm.T3[a, b, e] * (ub[0][0] * ue[1] + ub[1][0] * ue[2])
                loc = np.einsum("cq,iq,q->ci", integrand, self.Vv, self.wq2)
                vec = np.zeros(nv2)
                np.add.at(vec, self.cell_vnodes.ravel(), loc.ravel())
                r[c * nv2:(c + 1) * nv2] += dt * cv * vec
            Fn[a] = r
        Fn -= self.forcing_vector(n)
        Fn = Fn.ravel()
        mask = np.tile(self.spatial_dirichlet(), self.nt)
        g = self.boundary_values()[self.block(n, 0):self.block(n + 1, 0)]
        Un = Un.ravel()
        Fn[mask] = Un[mask] - g[mask]
        return Fn

    def slab_blocks(self, W, slab):
        """(diagonal block, subdiagonal block) of J(W) for ``slab`` before the
        Dirichlet elimination, as sparse matrices over ((q+1) S) x ((q+1) S)."""
        tm, dt, nu, cv = self.tm, self.dt, self.pb.nu, self.pb.conv
        Wn = self._slab(W, slab)
        D = sp.kron(tm.Kt, self.Mv) + dt * (nu * sp.kron(tm.Wt, self.Kv) + sp.kron(tm.Wt, self.G))
        for c in range(self.nt):
            D = D + dt * cv * sp.kron(tm.T3[:, :, c], self.convection_matrix(Wn[c]))
        E = np.zeros((self.nt, self.nt))
        E[:, self.nt - 1] = -tm.tau0
        L = sp.kron(E, self.Mv)
        return D.tocsr(), L.tocsr()

    def local_slab_blocks(self, W, slab, cells):
        """``slab_blocks`` assembled over the cells with ids in ``cells`` only: the
        space-time problem restricted to those cells (used for the patch matrix
        assembled over a patch's own cells)."""
        tm, dt, nu, cv = self.tm, self.dt, self.pb.nu, self.pb.conv
        Wn = self._slab(W, slab)
        Mv, Kv, G = self.linear_matrices_on(cells)
        D = sp.kron(tm.Kt, Mv) + dt * (nu * sp.kron(tm.Wt, Kv) + sp.kron(tm.Wt, G))
        for c in range(self.nt):
            D = D + dt * cv * sp.kron(tm.T3[:, :, c], self.convection_matrix(Wn[c], cells))
        E = np.zeros((self.nt, self.nt))
        E[:, self.nt - 1] = -tm.tau0
        L = sp.kron(E, Mv)
        return D.tocsr(), L.tocsr()

    def jacobian(self, W):
        """Global J(W) (block lower bidiagonal in slabs, Newton linearisation of the
        convection) with Dirichlet rows and columns replaced by the identity."""
        N = self.N
        blocks = [[None] * N for _ in range(N)]
        for n in range(N):
            D, L = self.slab_blocks(W, n)
            blocks[n][n] = D
            if n > 0:
                blocks[n][n - 1] = L
        J = sp.bmat(blocks, format="csr")
        mask = self.dirichlet_mask()
        Z = sp.diags((~mask).astype(np.float64))
        J = (Z @ J @ Z + sp.diags(mask.astype(np.float64))).tocsr()
        J.eliminate_zeros()
        return J

    def jacobian_slab(self, W, n):
        """(diagonal, subdiagonal) blocks of the rows of J(W) that belong to slab n,
        with the same Dirichlet elimination as ``jacobian``."""
        D, L = self.slab_blocks(W, n)
        m = np.tile(self.spatial_dirichlet(), self.nt)
        Z = sp.diags((~m).astype(np.float64))
        D = (Z @ D @ Z + sp.diags(m.astype(np.float64))).tocsr()
        L = (Z @ L @ Z).tocsr()
        return D, L

    def initial_guess(self):
        """Boundary lift at every temporal node, zero interior, zero pressure."""
        return self.boundary_values()

    def project_pressure(self, x):
        """Remove the mean int Phi of every temporal DoF's pressure (null space of J)."""
        x = x.copy()
        w = self.pressure_weights
        for blk in range(self.N * self.nt):
            off = blk * self.S + self.off_p
            p = x[off:off + self.np_ ** 2]
            x[off:off + self.np_ ** 2] = p - np.dot(w, p) / np.sum(w)
        return x
