"""Spatial grid transfers copied over every temporal DoF (oracle; test
infrastructure only).

Sec. 3: P = I (x) P_h with P_h = blockdiag(P_u, P_phi) the finite-element
interpolation from the 2h grid to the h grid, and R = P^T.  On the uniform
quadrilateral hierarchy P_u = P1_v (x) P1_v per velocity component and
P_phi = P1_p (x) P1_p, where P1[i_f, i_c] is the coarse 1D Lagrange basis
function i_c evaluated at fine node i_f.  Dirichlet rows and columns are zeroed
(corrections vanish on the Dirichlet boundary), so R = P^T holds exactly on the
free DoFs.
"""
import numpy as np
import scipy.sparse as sp

from .basis import equispaced_nodes, lagrange


def interpolation_1d(n_coarse, p):
    """1D matrix (n_f+1 ... ) from coarse Q_p on n_coarse cells to the mesh with 2 n_coarse cells."""
    nf_nodes = 2 * n_coarse * p + 1
    nc_nodes = n_coarse * p + 1
    P = np.zeros((nf_nodes, nc_nodes))
    ref = equispaced_nodes(p)
    hc = 1.0 / n_coarse
    for i_f in range(nf_nodes):
        x = i_f / (2.0 * n_coarse * p)
        cell = min(int(np.floor(x / hc)), n_coarse - 1)
        xi = x / hc - cell
        V, _ = lagrange(ref, [xi])
        for a in range(p + 1):
            P[i_f, cell * p + a] += V[a, 0]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def prolongation(fine, coarse):
    """Sparse global P from the coarse level's vectors to the fine level's."""
    Ph = spatial_prolongation(fine, coarse)
    return sp.kron(sp.identity(fine.N * fine.nt), Ph).tocsr()


def spatial_prolongation(fine, coarse):
    """P_h = blockdiag(P_u, P_u, P_phi) acting on one temporal block, Dirichlet rows and columns zero."""
    assert fine.n == 2 * coarse.n and fine.k == coarse.k and fine.q == coarse.q and fine.N == coarse.N
    k = fine.k
    P1v = sp.csr_matrix(interpolation_1d(coarse.n, k + 1))
    P1p = sp.csr_matrix(interpolation_1d(coarse.n, k))
    Pv = sp.kron(P1v, P1v)     # (y, x) ordering: kron(P_y, P_x)
    Pp = sp.kron(P1p, P1p)
    Ph = sp.block_diag([Pv, Pv, Pp]).tocsr()
    zf = sp.diags((~fine.spatial_dirichlet()).astype(np.float64))
    zc = sp.diags((~coarse.spatial_dirichlet()).astype(np.float64))
    Ph = (zf @ Ph @ zc).tocsr()
    Ph.eliminate_zeros()
    return Ph


def injection(fine, coarse, W):
    """Coarse-level iterate: the fine iterate at the coarse nodes (nested
    equispaced nodes, so the coarse node I is fine node 2I)."""
    out = np.zeros(coarse.ndofs)
    nvf, nvc = fine.nv, coarse.nv
    npf, npc = fine.np_, coarse.np_
    for blk in range(fine.N * fine.nt):
        fo, co = blk * fine.S, blk * coarse.S
        for c in range(2):
            u = W[fo + c * nvf * nvf:fo + (c + 1) * nvf * nvf].reshape(nvf, nvf)
            out[co + c * nvc * nvc:co + (c + 1) * nvc * nvc] = u[::2, ::2].ravel()
        p = W[fo + fine.off_p:fo + fine.S].reshape(npf, npf)
        out[co + coarse.off_p:co + coarse.S] = p[::2, ::2].ravel()
    return out
