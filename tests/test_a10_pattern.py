"""The sparsity of the off-diagonal temporal block A10 of a DG(1) patch block (CPU).

Of the four blocks the DG(1) slab solve stores per (patch, slab), A10 is not a factor but
the assembled block of the space-time Jacobian that couples the slab's second temporal
DoF to its first.  The FP64 smoother stores and applies it only on the slot pairs that
share a cell of the patch's 2 x 2 cells (and are not both pressure slots), and the bench
counts exactly those pairs as its algorithmic work.  This pins that rule to the oracle's
assembled Jacobian: on every patch and slab of small Q2/Q1 and Q3/Q2 meshes, with the
Newton convection about a random iterate, A10 has no nonzero outside the pattern, the
pattern is not loose, and an interior patch has the pair counts the kernels' segment
tables are built for (4744 of 107^2 for Q3/Q2, 1256 of 51^2 for Q2/Q1).
"""
import numpy as np
import pytest

import bench
from oracle.fem import Discretisation
from oracle.patches import patch_dofs
from paper_2407_13997_gb300 import inputs
from tests.oracle_problems import oracle_problem


@pytest.mark.parametrize("k,interior_pairs", [(1, 1256), (2, 4744)])
def test_a10_nonzeros_lie_in_the_cell_sharing_pattern(k, interior_pairs):
    n = 4
    w = inputs.fourier_small(n=n, k=k, q=1, N=2, nu=0.02)
    d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
    rng = np.random.default_rng(4)
    W = 0.5 * rng.standard_normal(d.ndofs)
    mask = d.dirichlet_mask()
    W[mask] = d.boundary_values()[mask]
    J = d.jacobian(W).tocsr()
    nnz = pairs = 0
    for p in range((n + 1) ** 2):
        for slab in range(w.N):
            idx = patch_dofs(d, p, slab)
            m = len(idx) // 2
            A10 = J[idx[m:]][:, idx[:m]].toarray()  # rows: temporal DoF 1, columns: temporal DoF 0
            pat = bench._a10_pattern(w, p, idx[:m] - d.block(slab, 0))
            assert pat.shape == A10.shape
            assert not np.any((A10 != 0) & ~pat), (p, slab)
            nnz += np.count_nonzero(A10)
            pairs += int(pat.sum())
    assert nnz > 0.9 * pairs, (nnz, pairs)  # the pattern is the coupling, not a loose bound
    centre = (n // 2) * (n + 1) + n // 2  # all slots of the centre patch are real
    sp = patch_dofs(d, centre, 0)
    assert bench._a10_nonzeros(w, centre, sp[:len(sp) // 2]) == interior_pairs
