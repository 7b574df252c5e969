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
