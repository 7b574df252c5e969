"""Pins for the oracle's solver layers (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import Discretisation, Problem
from oracle.solver import (CoarseSolver, Hierarchy, Options, arnoldi_ritz_max, chebyshev, fgmres,
                           newton_solve, splitmix64_raw, splitmix64_uniform, timestepping_solve)
from tests.test_oracle_fem import direct_solve


def test_splitmix64_matches_published_sequence():
    # reference outputs of splitmix64 from state 0
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in splitmix64_raw(0, 4)] == ref
    u = splitmix64_uniform(3, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


@pytest.mark.parametrize("zero_guess", [True, False])
def test_chebyshev_error_is_scaled_chebyshev_polynomial(zero_guess):
    """For J = diag(l_i), M = I, two steps on [a, b] give e_2 = T_2((theta - l)/delta)
    / T_2(theta/delta) e_0 with T_2(t) = 2t^2 - 1 (closed form)."""
    lam_est = 2.0
    opts = Options()
    a, b = 0.25 * lam_est, 1.05 * lam_est
    theta, delta = (a + b) / 2, (b - a) / 2
    lams = np.linspace(0.1, 2.1, 41)
    rng = np.random.default_rng(0)
    xstar = rng.standard_normal(lams.size)
    rhs = lams * xstar
    x0 = None if zero_guess else rng.standard_normal(lams.size)
    e0 = xstar - (0.0 if x0 is None else x0)
    x = chebyshev(lambda v: lams * v, lambda v: v.copy(), rhs, x0, lam_est, opts)
    T2 = lambda t: 2 * t * t - 1
    expect = T2((theta - lams) / delta) / T2(theta / delta) * e0
    assert np.abs((xstar - x) - expect).max() < 1e-13


def test_arnoldi_ritz_values():
    rng = np.random.default_rng(1)
    lam = np.array([0.5, 1.0, 1.5, 2.0, 3.0, 3.5, 4.0, 7.0, 7.5, 9.0])
    assert abs(arnoldi_ritz_max(lambda v: lam * v, rng.standard_normal(10), 10) - 9.0) < 1e-10
    # non-normal block with complex pair 5 +- 2i and real eigenvalue 4: largest real part 5
    A = np.array([[5.0, 2.0, 1.0], [-2.0, 5.0, 0.3], [0.0, 0.0, 4.0]])
    assert abs(arnoldi_ritz_max(lambda v: A @ v, rng.standard_normal(3), 3) - 5.0) < 1e-10


def test_coarse_solve_solves_consistent_systems_exactly():
    mx = np.array([1, 2]); my = np.array([1, 1]); amp = np.array([0.5, -0.2])
    d = Discretisation(2, 2, 1, 3, Problem(kind="fourier", nu=0.01, conv=1.0, T=0.3, mx=mx, my=my, amp=amp))
    rng = np.random.default_rng(3)
    W = rng.standard_normal(d.ndofs)
    J = d.jacobian(W)
    x = rng.standard_normal(d.ndofs) * ~d.dirichlet_mask()
    x = d.project_pressure(x)
    cs = CoarseSolver(d, J)
    y = cs.solve(J @ x)
    assert np.abs(y - x).max() < 1e-10 * np.abs(x).max()


def test_fgmres_against_dense_solve():
    rng = np.random.default_rng(4)
    A = np.eye(60) * 4 + rng.standard_normal((60, 60)) * 0.3
    b = rng.standard_normal(60)
    x, its = fgmres(lambda v: A @ v, lambda v: v.copy(), b, 1e-13 * np.linalg.norm(b), restart=30)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    Ainv = np.linalg.inv(A)
    x, its = fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-10 * np.linalg.norm(b))
    assert its == 1


def test_newton_wrmg_converges_to_the_direct_space_time_solution():
    """The brute-force Newton with sparse direct solves and the Newton-FGMRES-WRMG
    iteration must reach the same discrete solution (run to 1e-12)."""
    pb = Problem(kind="taylor_green", nu=0.02, conv=1.0, T=0.5)
    h = Hierarchy(4, 2, 1, 1, 3, pb, Options(newton_rtol=1e-12))
    st = {}
    U = newton_solve(h, stats=st)
    ref = direct_solve(h.fine, tol=1e-13)
    assert np.abs(U - ref).max() < 1e-10 * np.abs(ref).max()
    assert st["residuals"][-1] <= 1e-12 * st["residuals"][0]


def test_multigrid_iterations_are_mesh_independent():
    """FGMRES iterations per Newton step stay within +-2 as the mesh is refined."""
    its = []
    for n in (4, 8, 16):
        pb = Problem(kind="taylor_green", nu=0.01, conv=1.0, T=0.5)
        h = Hierarchy(n, 2, 1, 0, 2, pb, Options(ew=False, eta_fixed=1e-6, newton_maxit=1))
        st = {}
        newton_solve(h, stats=st)
        its.append(st["gmres"][0])
    assert max(its) - min(its) <= 2, its


def test_taylor_green_config_solves_to_tolerance_and_is_accurate():
    """8x8 Q2/Q1, DG(0), 8 slabs, nu = 1e-2: converges to 1e-8 and the end
    velocity is within the O(dt) DG(0) error of the exact Taylor-Green vortex."""
    pb = Problem(kind="taylor_green", nu=1e-2, conv=1.0, T=1.0)
    h = Hierarchy(8, 2, 1, 0, 8, pb)
    st = {}
    U = newton_solve(h, stats=st)
    d = h.fine
    assert st["residuals"][-1] <= 1e-8 * st["residuals"][0]
    assert len(st["gmres"]) <= 6
    ex = d.interpolant()
    off = d.block(d.N - 1, 0)
    err = np.abs(U[off:off + d.off_p] - ex[off:off + d.off_p]).max()
    assert err < 0.02, err


@pytest.mark.parametrize("kind,k,q", [("taylor_green", 1, 1), ("poly", 2, 1), ("taylor_green", 1, 0)])
def test_timestepping_reaches_the_all_at_once_solution(kind, k, q):
    """The space-time system is block lower bidiagonal in slabs (causal), so solving
    slab after slab with the previous end state as initial data must give the
    all-at-once discrete solution; the time offset enters the boundary data (Taylor-
    Green) and the forcing (poly), the end state the jump.  Both are taken from the
    brute-force direct Newton of the whole space-time system."""
    pb = Problem(kind=kind, nu=0.05, conv=1.0, T=0.6)
    N = 3
    ref = direct_solve(Discretisation(4, k, q, N, pb), tol=1e-13)
    U = timestepping_solve(4, 2, k, q, N, pb, Options(newton_rtol=1e-13, ew=False, eta_fixed=1e-12))
    assert np.abs(U - ref).max() < 1e-9 * np.abs(ref).max()
    # the first step alone is the one-slab problem on [0, T/N] with the exact initial data
    d1 = Discretisation(4, k, q, 1, Problem(kind=kind, nu=0.05, conv=1.0, T=0.2))
    first = direct_solve(d1, tol=1e-13)
    assert np.abs(U[:d1.ndofs] - first).max() < 1e-9 * np.abs(first).max()


def test_shifted_problem_uses_its_start_time():
    """A one-slab problem starting at t0 has the boundary data and the initial state
    of the exact Taylor-Green solution at t0 and its nodes (closed form)."""
    pb = Problem(kind="taylor_green", nu=0.05, conv=1.0, T=0.2, t0=0.4)
    d = Discretisation(4, 1, 1, 1, pb)
    xv, _ = d.node_coords()
    X, Y = np.meshgrid(xv, xv, indexing="xy")
    e = np.exp(-2 * 0.05 * np.pi ** 2 * 0.4)
    u0 = d.initial_velocity()
    assert np.allclose(u0[:d.nv ** 2], (-np.cos(np.pi * X) * np.sin(np.pi * Y) * e).ravel(), atol=1e-15)
    assert np.allclose(d.time_nodes(0), 0.4 + 0.2 * d.tm.nodes)


def test_newton_gives_up_on_divergence_and_on_fgmres_stagnation():
    """The safeguards stop Newton early: a divergence tolerance below 1 stops before
    the first step; an FGMRES limit of one iteration exhausts every inner solve, so
    Newton stops after `newton_stall` steps."""
    pb = Problem(kind="taylor_green", nu=0.02, conv=1.0, T=0.5)
    st = {}
    newton_solve(Hierarchy(4, 2, 1, 0, 2, pb, Options(newton_divtol=0.5)), stats=st)
    assert st["gmres"] == []
    st = {}
    newton_solve(Hierarchy(4, 2, 1, 0, 2, pb, Options(gmres_maxit=1, newton_stall=2)), stats=st)
    assert st["gmres"] == [1, 1]
    st = {}
    U = newton_solve(Hierarchy(4, 2, 1, 0, 2, pb, Options()), stats=st)
    assert st["residuals"][-1] <= 1e-8 * st["residuals"][0]
