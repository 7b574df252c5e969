"""Pins for the oracle's Vanka+star patches and waveform patch solve (CPU only)."""
import numpy as np
import pytest

from oracle.fem import Discretisation, Problem
from oracle.patches import PatchSmoother, patch_dofs, patch_spatial_indices
from paper_2407_13997_gb300.inputs import fourier_forcing


def disc(n, k, q, N):
    mx, my, amp = fourier_forcing(5)
    return Discretisation(n, k, q, N, Problem(kind="fourier", nu=0.02, conv=1.0, T=0.5,
                                              mx=mx, my=my, amp=amp))


def geometric_patch(d, I, J):
    """The patch from its geometric definition: velocity nodes in the closed
    2x2-cell block around vertex (I, J) off the Dirichlet boundary; pressure
    nodes strictly inside the block (the open star)."""
    h = d.h
    xv, xp = d.node_coords()
    lo_x, hi_x, lo_y, hi_y = (I - 1) * h, (I + 1) * h, (J - 1) * h, (J + 1) * h
    eps = 1e-12
    idx = []
    for c in range(2):
        for gy, y in enumerate(xv):
            for gx, x in enumerate(xv):
                inside = lo_x - eps <= x <= hi_x + eps and lo_y - eps <= y <= hi_y + eps
                interior = 0 < gx < d.nv - 1 and 0 < gy < d.nv - 1
                if inside and interior:
                    idx.append(c * d.nv ** 2 + gy * d.nv + gx)
    for py, y in enumerate(xp):
        for px, x in enumerate(xp):
            if lo_x + eps < x < hi_x - eps and lo_y + eps < y < hi_y - eps:
                idx.append(d.off_p + py * d.np_ + px)
    return np.array(idx)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_patch_index_lists_match_geometric_definition(k):
    d = disc(4, k, 0, 1)
    for J in range(d.n + 1):
        for I in range(d.n + 1):
            assert np.array_equal(patch_spatial_indices(d, I, J), geometric_patch(d, I, J))


@pytest.mark.parametrize("k,q", [(1, 0), (1, 1), (2, 1), (2, 0)])
def test_interior_patch_size_and_coverage(k, q):
    """Interior patch: (q+1) * (2 (2k+3)^2 + (2k-1)^2) DoFs -- 51 (q+1) for Q2/Q1
    and 107 (q+1) for Q3/Q2 -- and every free DoF lies in some patch."""
    d = disc(4, k, q, 2)
    m = (q + 1) * (2 * (2 * k + 3) ** 2 + (2 * k - 1) ** 2)
    assert len(patch_dofs(d, 2 * (d.n + 1) + 2, 1)) == m
    assert m == {1: 51, 2: 107}[k] * (q + 1)
    covered = np.zeros(d.ndofs, dtype=bool)
    for i in range((d.n + 1) ** 2):
        for s in range(d.N):
            ix = patch_dofs(d, i, s)
            assert len(np.unique(ix)) == len(ix)
            covered[ix] = True
    assert np.array_equal(covered, ~d.dirichlet_mask())


@pytest.mark.parametrize("n,k,q,N", [(2, 1, 0, 3), (3, 1, 1, 2), (2, 2, 1, 2), (4, 1, 0, 2)])
def test_smoother_equals_sum_of_explicit_space_time_patch_inverses(n, k, q, N):
    """M^{-1} r = sum_i R_i^T inv(J[P_i, P_i]) R_i r with the whole space-time
    patch (all slabs at once) inverted densely: pins the forward substitution
    over slabs (Eq. waveform_patch_solve) and the additive scatter."""
    d = disc(n, k, q, N)
    rng = np.random.default_rng(11)
    W = rng.standard_normal(d.ndofs)
    J = d.jacobian(W)
    sm = PatchSmoother(d, J)
    r = rng.standard_normal(d.ndofs)
    ref = np.zeros(d.ndofs)
    for i in range((n + 1) ** 2):
        ix = np.concatenate([patch_dofs(d, i, s) for s in range(N)])
        ref[ix] += np.linalg.inv(J[ix][:, ix].toarray()) @ r[ix]
    out = sm.apply(r)
    assert np.abs(out - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.all(out[d.dirichlet_mask()] == 0.0)
    w = rng.uniform(0.5, 1.0, d.ndofs)
    ref_w = np.zeros(d.ndofs)
    for i in range((n + 1) ** 2):
        ix = np.concatenate([patch_dofs(d, i, s) for s in range(N)])
        ref_w[ix] += w[ix] * (np.linalg.inv(J[ix][:, ix].toarray()) @ r[ix])
    assert np.abs(sm.apply(r, w) - ref_w).max() < 1e-10 * np.abs(ref_w).max()


@pytest.mark.parametrize("k,q", [(1, 0), (2, 1)])
def test_cell_restricted_assembly_sums_to_the_global_slab_blocks(k, q):
    """Assembly is a sum over cells: the slab blocks assembled over all cells, and
    the sum of those assembled over the two halves of any partition of the cells,
    equal the global slab blocks (pins the cell restriction of reading (B))."""
    from oracle.patches import patch_cells  # noqa: F401  (module under test)
    d = disc(3, k, q, 2)
    rng = np.random.default_rng(4)
    W = rng.standard_normal(d.ndofs)
    D, L = d.slab_blocks(W, 1)
    cells = np.arange(d.n * d.n)
    Da, La = d.local_slab_blocks(W, 1, cells)
    assert abs(Da - D).max() < 1e-13 * abs(D).max() and abs(La - L).max() < 1e-13 * abs(L).max()
    part = rng.permutation(cells)
    D1, L1 = d.local_slab_blocks(W, 1, part[:4])
    D2, L2 = d.local_slab_blocks(W, 1, part[4:])
    assert abs(D1 + D2 - D).max() < 1e-13 * abs(D).max()
    assert abs(L1 + L2 - L).max() < 1e-13 * abs(L).max()


def test_local_patch_matrix_equals_submatrix_when_the_patch_covers_the_mesh():
    """On the 2x2 mesh the centre vertex's 2x2 cell block is the whole mesh, so the
    patch system assembled over the patch's cells (reading (B)) is the principal
    submatrix (reading (A)); other patches differ."""
    d = disc(2, 1, 1, 3)
    rng = np.random.default_rng(5)
    W = rng.standard_normal(d.ndofs)
    J = d.jacobian(W)
    a = PatchSmoother(d, J)
    b = PatchSmoother(d, J, local=True, W=W)
    r = rng.standard_normal(d.ndofs)
    ya, yb = a.patch_solve(4, r), b.patch_solve(4, r)
    for s in range(d.N):
        assert np.abs(ya[s] - yb[s]).max() < 1e-12 * np.abs(ya[s]).max()
    y0a, y0b = a.patch_solve(0, r), b.patch_solve(0, r)
    assert np.abs(y0a[0] - y0b[0]).max() > 1e-6 * np.abs(y0a[0]).max()


@pytest.mark.parametrize("k", [1, 2])
def test_local_and_submatrix_patch_blocks_differ_only_on_boundary_velocity_pairs(k):
    """For an interior patch the two readings differ only through the cells outside
    the 2x2 block, i.e. on pairs of velocity DoFs that both lie on the boundary of
    the block; pressure rows and columns and interior velocity rows agree."""
    d = disc(4, k, 0, 1)
    rng = np.random.default_rng(6)
    W = rng.standard_normal(d.ndofs)
    J = d.jacobian(W)
    I = Jv = 2
    patch = Jv * (d.n + 1) + I
    ix = patch_dofs(d, patch, 0)
    A = J[ix][:, ix].toarray()
    from oracle.patches import patch_cells
    D, _ = d.local_slab_blocks(W, 0, patch_cells(d, patch))
    B = D[ix][:, ix].toarray()
    nv2 = d.nv ** 2
    lo, hi = (I - 1) * (k + 1), (I + 1) * (k + 1)

    def on_boundary(g):
        if g >= d.off_p:
            return False
        s = g % nv2
        gx, gy = s % d.nv, s // d.nv
        return gx in (lo, hi) or gy in (lo, hi)

    bnd = np.array([on_boundary(g) for g in ix])
    diff = np.abs(A - B) > 1e-13 * np.abs(A).max()
    assert diff.any()
    assert not (diff & ~np.outer(bnd, bnd)).any()


@pytest.mark.parametrize("k", [1, 2])
def test_multiplicity_weights_closed_form(k):
    """A velocity node at a mesh-vertex position along one direction lies in the
    closed blocks of 3 patches, one inside a cell in 2; a pressure node at a vertex
    position lies in the open star of 1 patch, one inside a cell in 2.  The count
    is the product over the two directions."""
    from oracle.patches import multiplicity_weights
    d = disc(4, k, 1, 2)
    w = multiplicity_weights(d)
    free = ~d.dirichlet_mask()
    expect = np.zeros(d.ndofs)
    for slab in range(d.N):
        for a in range(d.nt):
            base = d.block(slab, a)
            for c in range(2):
                for gy in range(d.nv):
                    for gx in range(d.nv):
                        mv = lambda g: 3 if g % (k + 1) == 0 else 2
                        expect[base + d.vel_index(c, gx, gy)] = 1.0 / (mv(gx) * mv(gy))
            for py in range(d.np_):
                for px in range(d.np_):
                    mp = lambda g: 1 if g % k == 0 else 2
                    expect[base + d.pres_index(px, py)] = 1.0 / (mp(px) * mp(py))
    assert np.allclose(w[free], expect[free], rtol=0, atol=1e-15)
    assert np.all(w[~free] == 0.0)
