"""Pins for the oracle's heat-equation waveform relaxation (CPU only)."""
import os
from math import factorial

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle.fem import Discretisation, Problem
from oracle.heat import (HeatDiscretisation, HeatHierarchy, HeatProblem, HeatSmoother, global_1d, heat_patch_dofs,
                         heat_patch_spatial, heat_solve)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")


def paper_dof_counts():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append((f[0], int(f[1]), int(f[2]), int(f[3]), float(f[4])))
    return rows


@pytest.mark.parametrize("row", paper_dof_counts(), ids=lambda r: f"{r[0]}_k{r[1]}_q{r[2]}_N{r[3]}")
def test_dof_counts_match_the_papers_tables(row):
    """Tables heat:dof_nnz3 and chorin:dofs (Mref = 3: 80 x 80 cells), as printed to two
    significant digits."""
    kind, k, q, N, printed = row
    if kind == "heat":
        nd = HeatDiscretisation(80, k, q, N, HeatProblem()).ndofs
    else:
        nd = Discretisation(80, k, q, N, Problem()).ndofs
    assert float(f"{nd:.1e}") == printed, (nd, printed)


def pade(j, k, z):
    """(j, k) Pade approximant of exp(z), closed form."""
    num = sum(factorial(j + k - i) * factorial(j) / (factorial(j + k) * factorial(i) * factorial(j - i)) * z ** i
              for i in range(j + 1))
    den = sum(factorial(j + k - i) * factorial(k) / (factorial(j + k) * factorial(i) * factorial(k - i)) * (-z) ** i
              for i in range(k + 1))
    return num / den


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_discrete_eigenvector_decays_by_the_radau_stability_function(q):
    """u(0) = v with K v = mu M v (a discrete Neumann eigenvector): the space-time
    solution is U_{n,a} = c_{n,a} v, and its end value after N slabs is R(z)^N v with
    z = -nu mu dt and R the (q, q+1) Pade approximant of exp (DG(q) in time is Radau
    IIA on linear problems).  Exact to roundoff, for every degree in time."""
    pb = HeatProblem(nu=0.5, T=0.4)
    N = 4
    d = HeatDiscretisation(4, 2, q, N, pb)
    mu, V = sla.eigh(d.K.toarray(), d.M.toarray())
    for j in (1, 6, 20):
        v = V[:, j] / np.abs(V[:, j]).max()
        d.initial_state = v
        U = spla.spsolve(d.jacobian().tocsc(), d.rhs())
        end = U[d.block(N - 1, d.nt - 1):d.block(N - 1, d.nt - 1) + d.S]
        expect = pade(q, q + 1, -pb.nu * mu[j] * d.dt) ** N * v
        assert np.abs(end - expect).max() < 1e-11 * max(np.abs(expect).max(), 1e-3), (q, j)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_spatial_matrices_integrate_polynomials_exactly(k):
    """Q_k reproduces polynomials of degree k in each variable: 1^T M 1 = |Omega| = 1,
    K 1 = 0, x^T K x = int |grad x|^2 = 1, 1^T M x^k = 1/(k+1), and
    (x y)^T K (x y) = int (y^2 + x^2) = 2/3."""
    d = HeatDiscretisation(4, k, 0, 1, HeatProblem())
    x = d.node_coords()
    X, Y = np.meshgrid(x, x, indexing="xy")
    one = np.ones(d.S)
    assert abs(one @ d.M @ one - 1.0) < 1e-13
    assert np.abs(d.K @ one).max() < 1e-12
    xv = X.ravel()
    assert abs(xv @ d.K @ xv - 1.0) < 1e-12
    assert abs(one @ d.M @ xv ** k - 1.0 / (k + 1)) < 1e-13
    xy = (X * Y).ravel()
    assert abs(xy @ d.K @ xy - 2.0 / 3.0) < 1e-12
    M1, K1 = global_1d(3, k)
    assert np.allclose(M1, M1.T) and np.allclose(K1, K1.T)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_vertex_star_patches_are_open_stars(k):
    """Interior patch: (2k-1)^2 nodes strictly inside the 2x2 cell block; boundary
    vertices keep the boundary nodes of their star; every node lies in a patch."""
    d = HeatDiscretisation(4, k, 1, 2, HeatProblem())
    x = d.node_coords()
    h = 1.0 / d.n
    covered = np.zeros(d.S, dtype=bool)
    for J in range(d.n + 1):
        for I in range(d.n + 1):
            idx = heat_patch_spatial(d, I, J)
            geo = [gy * d.nv + gx for gy in range(d.nv) for gx in range(d.nv)
                   if (I - 1) * h + 1e-12 < x[gx] < (I + 1) * h - 1e-12
                   and (J - 1) * h + 1e-12 < x[gy] < (J + 1) * h - 1e-12]
            assert np.array_equal(idx, geo)
            covered[idx] = True
    assert len(heat_patch_spatial(d, 2, 2)) == (2 * k - 1) ** 2
    assert covered.all()


@pytest.mark.parametrize("q", [0, 1])
def test_eigenfunction_decay_converges(q):
    """u0 = cos(pi x) is a Neumann eigenfunction: u = exp(-nu pi^2 t) cos(pi x).  With a
    fine Q3 mesh the end-value error is the time error, O(dt^(2q+1)) (Radau IIA)."""
    errs = []
    for N in (4, 8):
        pb = HeatProblem(nu=1.0, T=0.2, u0="cos")
        d = HeatDiscretisation(8, 3, q, N, pb)
        U = spla.spsolve(d.jacobian().tocsc(), d.rhs())
        end = U[d.block(N - 1, d.nt - 1):d.block(N - 1, d.nt - 1) + d.S]
        x = d.node_coords()
        X, Y = np.meshgrid(x, x, indexing="xy")
        errs.append(np.abs(end - pb.exact(X, Y, 0.2).ravel()).max())
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - (2 * q + 1)) < 0.35, (errs, rate)


@pytest.mark.parametrize("n,k,q,N", [(2, 1, 0, 3), (2, 2, 1, 2), (4, 1, 1, 2), (2, 1, 2, 2), (2, 2, 3, 2)])
def test_smoother_equals_sum_of_explicit_space_time_patch_inverses(n, k, q, N):
    d = HeatDiscretisation(n, k, q, N, HeatProblem())
    J = d.jacobian()
    sm = HeatSmoother(d, J)
    r = np.random.default_rng(3).standard_normal(d.ndofs)
    ref = np.zeros(d.ndofs)
    for i in range((n + 1) ** 2):
        ix = np.concatenate([heat_patch_dofs(d, i, s) for s in range(N)])
        ref[ix] += np.linalg.inv(J[ix][:, ix].toarray()) @ r[ix]
    assert np.abs(sm.apply(r) - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("k,q,nc", [(1, 0, 2), (2, 1, 2), (3, 1, 2), (1, 2, 2), (2, 3, 2), (3, 3, 1)])
def test_fgmres_wrmg_reaches_the_direct_solution_in_few_iterations(k, q, nc):
    """FGMRES preconditioned by one WRMG V(2,2) cycle reaches the direct space-time
    solution; the paper reports 3 iterations to 1e-6 for its heat problems (4 for one
    case), across temporal degrees 0..3 and spatial degrees 1..3."""
    hier = HeatHierarchy(8, nc, k, q, 20, HeatProblem(nu=1.0, T=0.02))
    U, its = heat_solve(hier, rtol=1e-6, atol=1e-6)
    b = hier.fine.rhs()
    ref = spla.spsolve(hier.J[-1].tocsc(), b)
    # the stopping test, checked on the true residual
    assert np.linalg.norm(b - hier.J[-1] @ U) <= 1.001 * max(1e-6 * np.linalg.norm(b), 1e-6)
    assert its <= 5, its   # the paper reports 3 on its triangle meshes
    U2, its2 = heat_solve(hier, rtol=1e-12, atol=0.0)
    assert np.abs(U2 - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_all_at_once_equals_slab_by_slab_solves(q):
    """Causality of DG(q) in time (Eq. dgintime): the space-time system is block lower
    bidiagonal, so its solution equals N one-slab solves, each started from the
    previous slab's end value (the last temporal DoF, the right-Radau point s = 1)."""
    pb = HeatProblem(nu=0.7, T=0.3)
    N = 3
    d = HeatDiscretisation(4, 2, q, N, pb)
    U = spla.spsolve(d.jacobian().tocsc(), d.rhs())
    state = None
    for n in range(N):
        one = HeatDiscretisation(4, 2, q, 1, HeatProblem(nu=0.7, T=0.3 / N))
        one.initial_state = state
        u1 = spla.spsolve(one.jacobian().tocsc(), one.rhs())
        blk = U[d.block(n, 0):d.block(n + 1, 0)]
        assert np.abs(u1 - blk).max() < 1e-12 * np.abs(blk).max(), (q, n)
        state = u1[one.block(0, one.nt - 1):one.block(0, one.nt - 1) + one.S]
