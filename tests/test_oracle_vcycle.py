"""Pins for the oracle's V-cycle composition (Algorithm Vcycle, Sec. 3) and for the
Fourier forcing field (CPU only).

The pieces a cycle is made of are pinned elsewhere (Chebyshev by its closed-form
error polynomial, the smoother by explicit patch inverses, the coarse solve by
exact solves of consistent systems, the transfers by polynomial reproduction and
adjointness).  These tests pin how the cycle puts them together:

* with no smoothing steps a two-level cycle is exactly the coarse-grid correction
  P A_c^{-1} P^T;
* a V(2,2) cycle is a linear map C whose error propagation I - C J factors as
  S (I - P C_c P^T J) S, with S = I - Q J the error operator of the Chebyshev
  smoother (Q its zero-guess map) and C_c the exact coarse solve (two levels) or
  the next coarser V-cycle (three levels);
* on the paper's Chorin problem (Sec. 5, Reynolds form, DG(0), Q2/Q1) the
  preconditioned FGMRES needs few iterations per Newton step, as the paper's
  iteration table reports (4 Newton steps, 11 FGMRES iterations in total at
  N = 10, 20, 40).

A cycle that skips the post-smoothing, restricts b instead of the residual,
starts a coarser level from a non-zero guess or adds the correction with the
wrong sign fails the factorisation test.
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.solver import Hierarchy, Options, chebyshev, newton_solve
from oracle.transfer import injection
from paper_2407_13997_gb300 import inputs
from tests.oracle_problems import oracle_problem


def _linearised(n_fine, n_coarse, k, q, N, pb, opts, seed):
    h = Hierarchy(n_fine, n_coarse, k, q, N, pb, opts)
    d = h.fine
    rng = np.random.default_rng(seed)
    W = d.initial_guess() + 0.3 * rng.standard_normal(d.ndofs) * ~d.dirichlet_mask()
    h.linearise(W)
    return h, W


def _fourier(nu=0.05, T=0.5):
    mx, my, amp = inputs.fourier_forcing(0)
    return Problem(kind="fourier", nu=nu, conv=1.0, T=T, mx=mx, my=my, amp=amp)


def _smoother_error(lev, opts):
    """v -> (I - Q J) v, Q the zero-guess Chebyshev(2) map of the level."""
    J = lev.J

    def S(v):
        return v - chebyshev(lambda x: J @ x, lev.smoother.apply, J @ v, None, lev.lam, opts)
    return S


@pytest.mark.parametrize("k,q", [(1, 0), (1, 1)])
def test_two_level_cycle_without_smoothing_is_the_coarse_grid_correction(k, q):
    opts = Options(cheb_steps=0)
    h, _ = _linearised(4, 2, k, q, 2, _fourier(), opts, seed=1)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(h.fine.ndofs)
    x = h.vcycle(b)
    P = h.P[1]
    expect = P @ h.coarse.solve(P.T @ b)
    assert np.abs(x - expect).max() <= 1e-12 * np.abs(expect).max()
    assert np.abs(expect).max() > 0.1


@pytest.mark.parametrize("k,q", [(1, 0), (1, 1)])
def test_two_level_v22_error_propagation_factorises(k, q):
    """C J v = v - S (I - P A_c^{-1} P^T J) S v for random v."""
    opts = Options()
    h, _ = _linearised(4, 2, k, q, 2, _fourier(), opts, seed=3)
    fine = h.levels[1]
    J, P = fine.J, h.P[1]
    S = _smoother_error(fine, opts)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(h.fine.ndofs)
        e1 = S(v)
        e2 = e1 - P @ h.coarse.solve(P.T @ (J @ e1))
        expect = v - S(e2)
        got = h.vcycle(J @ v)
        assert np.abs(got - expect).max() <= 1e-10 * np.abs(expect).max()
    # the pieces are not trivial: each smoothing and the correction change the error
    assert np.abs(e1 - v).max() > 1e-3 * np.abs(v).max()
    assert np.abs(e2 - e1).max() > 1e-3 * np.abs(v).max()


def test_three_level_v22_recurses_on_the_coarser_cycle():
    """On three levels the coarse-grid correction is the two-level V-cycle of the
    coarser pair (zero initial guess there, its own pre- and post-smoothing)."""
    opts = Options()
    pb = _fourier()
    h3, W = _linearised(8, 2, 1, 0, 2, pb, opts, seed=5)
    h2 = Hierarchy(4, 2, 1, 0, 2, pb, opts)
    h2.linearise(injection(h3.levels[2].disc, h3.levels[1].disc, W))
    # same level-1 operators and eigen-estimate in both hierarchies
    assert abs(h2.levels[1].lam - h3.levels[1].lam) <= 1e-12 * h3.levels[1].lam
    fine = h3.levels[2]
    J, P = fine.J, h3.P[2]
    S = _smoother_error(fine, opts)
    rng = np.random.default_rng(6)
    for _ in range(2):
        v = rng.standard_normal(h3.fine.ndofs)
        e1 = S(v)
        e2 = e1 - P @ h2.vcycle(P.T @ (J @ e1))
        expect = v - S(e2)
        got = h3.vcycle(J @ v)
        assert np.abs(got - expect).max() <= 1e-10 * np.abs(expect).max()


def test_chorin_fgmres_iterations_per_newton_step_are_small():
    """Sec. 5, Chorin problem (R = 10, t in [0, 0.1], Q2/Q1, DG(0), N = 10): the paper
    reports 4 Newton steps and 11 FGMRES iterations (2.75 per step) on its meshes.
    The oracle's cycle must be at least that effective on a small mesh: at most 6
    FGMRES iterations per Newton step on average and at most 6 Newton steps."""
    w = inputs.chorin(n=8, k=1, q=0, N=10)
    h = Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options())
    st = {}
    newton_solve(h, stats=st)
    assert st["residuals"][-1] <= 1e-8 * st["residuals"][0]
    steps = len(st["gmres"])
    assert steps <= 6, st["gmres"]
    assert sum(st["gmres"]) <= 6 * steps, st["gmres"]


def _stream(pb, x, y):
    return sum(a * np.sin(m * np.pi * x) * np.sin(n * np.pi * y) for m, n, a in zip(pb.mx, pb.my, pb.amp))


def test_fourier_forcing_is_the_curl_of_the_stream_function():
    """f = (d_y psi, -d_x psi) at random points, against central differences of psi."""
    pb = _fourier()
    rng = np.random.default_rng(7)
    x, y = rng.uniform(0.0, 1.0, 200), rng.uniform(0.0, 1.0, 200)
    eps = 1e-5
    dpsi_dx = (_stream(pb, x + eps, y) - _stream(pb, x - eps, y)) / (2 * eps)
    dpsi_dy = (_stream(pb, x, y + eps) - _stream(pb, x, y - eps)) / (2 * eps)
    fx, fy = pb.forcing(x, y, 0.3)
    scale = np.abs(np.concatenate([dpsi_dx, dpsi_dy])).max()
    assert np.abs(fx - dpsi_dy).max() <= 1e-7 * scale
    assert np.abs(fy + dpsi_dx).max() <= 1e-7 * scale
    # time-independent
    fx1, fy1 = pb.forcing(x, y, 0.9)
    assert np.array_equal(fx, fx1) and np.array_equal(fy, fy1)


def test_fourier_forcing_is_divergence_free_and_not_curl_free():
    pb = _fourier()
    rng = np.random.default_rng(8)
    x, y = rng.uniform(0.0, 1.0, 200), rng.uniform(0.0, 1.0, 200)
    eps = 1e-5
    dfx_dx = (pb.forcing(x + eps, y, 0)[0] - pb.forcing(x - eps, y, 0)[0]) / (2 * eps)
    dfy_dy = (pb.forcing(x, y + eps, 0)[1] - pb.forcing(x, y - eps, 0)[1]) / (2 * eps)
    dfy_dx = (pb.forcing(x + eps, y, 0)[1] - pb.forcing(x - eps, y, 0)[1]) / (2 * eps)
    dfx_dy = (pb.forcing(x, y + eps, 0)[0] - pb.forcing(x, y - eps, 0)[0]) / (2 * eps)
    scale = np.abs(np.concatenate([dfx_dx, dfy_dy])).max()
    assert np.abs(dfx_dx + dfy_dy).max() <= 1e-6 * scale
    # the curl of f is -lap psi, far from zero
    assert np.abs(dfy_dx - dfx_dy).max() > 0.1 * scale


def test_fourier_amplitudes_follow_the_stated_recipe():
    """The 8 lowest mode pairs ordered by (m^2 + n^2, m), amplitudes z_j / (m_j^2 + n_j^2)
    with z ~ N(0, 1) from numpy's default_rng(seed)."""
    pairs = sorted(((m, n) for m in range(1, 6) for n in range(1, 6)), key=lambda p: (p[0] ** 2 + p[1] ** 2, p[0]))
    mx, my, amp = inputs.fourier_forcing(11)
    assert list(zip(mx.tolist(), my.tolist())) == pairs[:8]
    z = np.random.default_rng(11).standard_normal(8)
    assert np.array_equal(amp, z / np.array([m * m + n * n for m, n in pairs[:8]], dtype=np.float64))
