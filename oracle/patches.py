"""Vanka+star space-time patches and the waveform patch solve (oracle; test
infrastructure only).

Patch definition (Sec. 3, NS relaxation; Fig. patches right): one patch per
mesh vertex (I, J).  It holds every velocity DoF in the closure of the vertex
star -- on a quadrilateral mesh the closure of the 2 x 2 cell block around the
vertex, (2k+3)^2 nodes per component -- and the pressure DoFs of the open star
(the vertex, the interiors of its 4 edges and of its 4 cells), (2k-1)^2 nodes.
Every spatial DoF is taken at all q+1 temporal DoFs of a slab and across all
slabs (the waveform extension).  Dirichlet and out-of-domain nodes are dropped
and the list is compacted.

Patch-local order, per slab: temporal DoF a outermost, then the u_x nodes
(y-major, x fastest), then u_y, then the pressure nodes.  Patch id = J*(n+1)+I.

Patch matrix: by default the principal submatrix A_i = J[P_i, P_i] of the
assembled space-time Jacobian (PCASM-style reading (A)); optionally (reading
(B)) the space-time Jacobian assembled over the patch's own 2 x 2 cells only,
restricted to P_i (subdiagonal included).  Because J is block lower
bidiagonal in slabs, the patch system is the block lower bidiagonal system of
Eq. waveform_patch_solve and is solved by forward substitution over slabs,
y_n = A_nn^{-1} (r_n - A_{n,n-1} y_{n-1}), each A_nn by dense LU with partial
pivoting.  The relaxation is M^{-1} r = sum_i R_i^T (w_i * A_i^{-1} R_i r),
w = 1 (plain additive) or w = 1 / (number of patches holding the DoF).
"""
import numpy as np
import scipy.linalg as sla


def patch_spatial_indices(disc, I, J):
    """Spatial (within one temporal block) indices of the patch at vertex (I, J)."""
    k, nv, np_ = disc.k, disc.nv, disc.np_
    dmask = disc.spatial_dirichlet()
    lo, hi = (I - 1) * (k + 1), (I + 1) * (k + 1)
    xs = [g for g in range(lo, hi + 1) if 0 <= g < nv]
    lo, hi = (J - 1) * (k + 1), (J + 1) * (k + 1)
    ys = [g for g in range(lo, hi + 1) if 0 <= g < nv]
    idx = []
    for c in range(2):
        for gy in ys:
            for gx in xs:
                s = disc.vel_index(c, gx, gy)
                if not dmask[s]:
                    idx.append(s)
    pxs = [p for p in range(I * k - (k - 1), I * k + (k - 1) + 1) if 0 <= p < np_]
    pys = [p for p in range(J * k - (k - 1), J * k + (k - 1) + 1) if 0 <= p < np_]
    for py in pys:
        for px in pxs:
            idx.append(disc.pres_index(px, py))
    return np.array(idx, dtype=np.int64)


def patch_dofs(disc, patch, slab):
    """Global indices of ``patch`` on ``slab``, in patch-local order."""
    n1 = disc.n + 1
    I, J = patch % n1, patch // n1
    sidx = patch_spatial_indices(disc, I, J)
    return np.concatenate([disc.block(slab, a) + sidx for a in range(disc.nt)])


def patch_cells(disc, patch):
    """Ids (J * n + I) of the cells of the 2 x 2 block around the patch's vertex."""
    n1 = disc.n + 1
    I, J = patch % n1, patch // n1
    return np.array([cy * disc.n + cx for cy in (J - 1, J) for cx in (I - 1, I)
                     if 0 <= cx < disc.n and 0 <= cy < disc.n], dtype=np.int64)


def multiplicity_weights(disc):
    """w = 1 / (number of patches whose index list holds the DoF); 0 on Dirichlet DoFs."""
    count = np.zeros(disc.ndofs)
    for i in range((disc.n + 1) ** 2):
        for s in range(disc.N):
            count[patch_dofs(disc, i, s)] += 1.0
    w = np.zeros(disc.ndofs)
    w[count > 0] = 1.0 / count[count > 0]
    return w


class PatchSmoother:
    """The waveform Vanka+star relaxation M^{-1} for one level's J.

    local=False: patch matrices are principal submatrices of J (reading (A));
    local=True: they are assembled over each patch's own cells about the
    iterate W (reading (B)); W is then required."""

    def __init__(self, disc, J, local=False, W=None):
        self.disc, self.J = disc, J
        self.npatch = (disc.n + 1) ** 2
        self.idx = [[patch_dofs(disc, i, s) for s in range(disc.N)] for i in range(self.npatch)]
        if not local:
            diag = [[J[ix][:, ix].toarray() for ix in row] for row in self.idx]
            sub = [[None] + [J[row[s]][:, row[s - 1]].toarray() for s in range(1, disc.N)] for row in self.idx]
        else:
            diag, sub = [], []
            for i, row in enumerate(self.idx):
                cells = patch_cells(disc, i)
                # patch indices within one slab's (q+1) S block
                loc = row[0] - disc.block(0, 0)
                drow, srow = [], [None]
                for s in range(disc.N):
                    D, L = disc.local_slab_blocks(W, s, cells)
                    drow.append(D[loc][:, loc].toarray())
                    if s > 0:
                        srow.append(L[loc][:, loc].toarray())
                diag.append(drow)
                sub.append(srow)
        # dense diagonal blocks A_nn factored by partial-pivot LU; subdiagonal blocks A_{n,n-1}
        self.lu = [[sla.lu_factor(A, check_finite=False) for A in row] for row in diag]
        self.sub = sub

    def patch_solve(self, i, r):
        """y_i = A_i^{-1} R_i r by forward substitution over slabs (Eq. waveform_patch_solve)."""
        ys = []
        for s in range(self.disc.N):
            rhs = r[self.idx[i][s]].copy()
            if s > 0:
                rhs -= self.sub[i][s] @ ys[-1]
            ys.append(sla.lu_solve(self.lu[i][s], rhs, check_finite=False))
        return ys

    def apply(self, r, weights=None):
        """M^{-1} r = sum_i R_i^T (w_i y_i); w = 1 unless ``weights`` (global) is given."""
        out = np.zeros_like(r)
        for i in range(self.npatch):
            ys = self.patch_solve(i, r)
            for s in range(self.disc.N):
                ix = self.idx[i][s]
                w = 1.0 if weights is None else weights[ix]
                np.add.at(out, ix, w * ys[s])
        return out
