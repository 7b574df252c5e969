"""Pins for the oracle's space-time discretisation (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.basis import gauss_legendre, lagrange
from oracle.fem import Discretisation, Problem
from paper_2407_13997_gb300.inputs import fourier_forcing


def fourier_problem(nu=0.05, conv=1.0, seed=3):
    mx, my, amp = fourier_forcing(seed)
    return Problem(kind="fourier", nu=nu, conv=conv, T=0.5, mx=mx, my=my, amp=amp)


@pytest.mark.parametrize("k,q,steady", [(1, 1, False), (1, 0, True), (2, 1, False), (2, 0, True), (1, 2, False)])
def test_manufactured_polynomial_solution_has_zero_residual(k, q, steady):
    """u = (y^2, x^2)(1+t), p = x+y-1 lies in the discrete space (k >= 1, q >= 1),
    is divergence free and is continuous in time, so with exact quadrature the
    interpolant (Phi = -p) must satisfy every equation of Eq. nsfem exactly."""
    pb = Problem(kind="poly", nu=0.3, conv=2.5, T=0.7, steady=steady)
    d = Discretisation(3, k, q, 2, pb)
    U = d.interpolant()
    F = d.residual(U)
    assert np.abs(F).max() < 1e-12
    # sensitivity: the wrong pressure sign leaves a residual
    U2 = U.copy()
    for blk in range(d.N * d.nt):
        U2[blk * d.S + d.off_p:(blk + 1) * d.S] *= -1.0
    assert np.abs(d.residual(U2)).max() > 1e-3


@pytest.mark.parametrize("k,q", [(1, 0), (1, 1), (2, 1)])
def test_jacobian_equals_central_difference_of_quadratic_residual(k, q):
    """F is quadratic in U, so (F(U + x) - F(U - x)) / 2 = J(U) x exactly for any
    x vanishing on the Dirichlet DoFs."""
    d = Discretisation(3, k, q, 3, fourier_problem())
    rng = np.random.default_rng(7)
    mask = d.dirichlet_mask()
    U = rng.standard_normal(d.ndofs)
    U[mask] = d.boundary_values()[mask]
    x = rng.standard_normal(d.ndofs)
    x[mask] = 0.0
    J = d.jacobian(U)
    fd = 0.5 * (d.residual(U + x) - d.residual(U - x))
    assert np.abs(fd - J @ x).max() < 1e-11 * np.abs(fd).max()


def test_jacobian_block_structure_and_jump_coupling():
    """J is block lower bidiagonal in slabs; the subdiagonal block is
    -tau_a(0) M_u acting on the last temporal DoF's velocity only (the DAE
    structure: pressure has no time derivative and no jump)."""
    d = Discretisation(3, 1, 1, 4, fourier_problem())
    U = np.random.default_rng(1).standard_normal(d.ndofs)
    J = d.jacobian(U).tocsr()
    B = (q1 := d.nt) * d.S
    free = ~d.spatial_dirichlet()
    for r in range(d.N):
        for c in range(d.N):
            blk = J[r * B:(r + 1) * B, c * B:(c + 1) * B]
            if c > r or c < r - 1:
                assert blk.nnz == 0
            if c == r - 1:
                blk = blk.toarray()
                for a in range(q1):
                    for b in range(q1):
                        sub = blk[a * d.S:(a + 1) * d.S, b * d.S:(b + 1) * d.S]
                        if b != q1 - 1:
                            assert np.abs(sub).max() == 0.0
                            continue
                        expect = -d.tm.tau0[a] * d.Mv.toarray()
                        expect[~free, :] = 0.0
                        expect[:, ~free] = 0.0
                        assert np.allclose(sub, expect, atol=1e-15)
                        assert np.abs(sub[:, d.off_p:]).max() == 0.0


def test_constant_pressure_is_null_vector_of_jacobian():
    d = Discretisation(4, 2, 1, 2, fourier_problem())
    U = np.random.default_rng(2).standard_normal(d.ndofs)
    J = d.jacobian(U)
    for blk in range(d.N * d.nt):
        x = np.zeros(d.ndofs)
        x[blk * d.S + d.off_p:(blk + 1) * d.S] = 1.0
        assert np.abs(J @ x).max() < 1e-13
        assert np.abs(J.T @ x).max() < 1e-13


def direct_solve(d, tol=1e-13, maxit=8):
    """Brute-force Newton with a sparse direct solve of the whole space-time system
    (one pressure DoF pinned per temporal DoF, then made mean-free)."""
    U = d.initial_guess()
    pins = [d.block(n, a) + d.pres_index(0, 0) for n in range(d.N) for a in range(d.nt)]
    F = d.residual(U)
    f0 = np.linalg.norm(F)
    for _ in range(maxit):
        if np.linalg.norm(F) <= tol * f0:
            break
        J = d.jacobian(U).tolil()
        rhs = -F
        for p in pins:
            J[p, :] = 0.0
            J[:, p] = 0.0
            J[p, p] = 1.0
            rhs[p] = 0.0
        U = U + d.project_pressure(spla.spsolve(sp.csc_matrix(J), rhs))
        F = d.residual(U)
    return U


@pytest.mark.parametrize("q,rate", [(0, 2.0), (1, 8.0)])
def test_end_point_error_converges_at_order_2q_plus_1(q, rate):
    """DG(q) in time = Radau IIA: for linear Stokes (conv = 0, Taylor-Green data,
    a genuine decay u_t = -2 nu pi^2 u) the end value converges at O(dt^{2q+1})
    towards the spatially semi-discrete solution, measured against N = 96 on the
    same mesh so that the spatial error cancels."""
    def end_value(N):
        pb = Problem(kind="taylor_green", nu=1.0 / np.pi ** 2, conv=0.0, T=0.25)
        d = Discretisation(2, 1, q, N, pb)
        U = direct_solve(d)
        off = d.block(N - 1, d.nt - 1)
        return U[off:off + d.off_p]
    ref = end_value(96)
    errs = [np.abs(end_value(N) - ref).max() for N in (3, 6, 12)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert abs(ratios[-1] / rate - 1.0) < 0.15, (errs, ratios)


@pytest.mark.parametrize("q", [0, 1])
def test_time_error_in_l2_converges_at_order_q_plus_1(q):
    """DG(q) in time: the L2-in-time error of the velocity converges at O(dt^{q+1}),
    the approximation order of degree-q polynomials in time.  Linear Stokes with
    Taylor-Green decay data; the error is measured against N = 192 slabs on the same
    mesh (so the spatial error cancels), with the DG polynomials evaluated at q+3
    Gauss points per slab."""
    pb = Problem(kind="taylor_green", nu=1.0 / np.pi ** 2, conv=0.0, T=0.25)

    def solve(N):
        d = Discretisation(2, 1, q, N, pb)
        return d, direct_solve(d)

    def velocity_at(d, U, t):
        n = min(int(t / d.dt), d.N - 1)
        V, _ = lagrange(d.tm.nodes, [t / d.dt - n])
        return sum(V[a, 0] * U[d.block(n, a):d.block(n, a) + d.off_p] for a in range(d.nt))

    dref, Uref = solve(192)
    xs, ws = gauss_legendre(q + 3)
    errs = []
    for N in (2, 4, 8):
        d, U = solve(N)
        e2 = 0.0
        for n in range(N):
            for x, wgt in zip(xs, ws):
                t = (n + x) * d.dt
                diff = velocity_at(d, U, t) - velocity_at(dref, Uref, t)
                e2 += wgt * d.dt * np.sum(diff ** 2)
        errs.append(np.sqrt(e2))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert abs(ratios[-1] / 2 ** (q + 1) - 1.0) < 0.15, (errs, ratios)


def l2_velocity_error(d, U, slab, a):
    """Spatial L2 error of the velocity at temporal DoF a of ``slab``."""
    t = d.time_nodes(slab)[a]
    off = d.block(slab, a)
    nv2 = d.nv ** 2
    err2 = 0.0
    ex = d.pb.exact_velocity(d.qpx, d.qpy, t)
    for c in range(2):
        uh = U[off + c * nv2:off + (c + 1) * nv2][d.cell_vnodes] @ d.Vv
        err2 += np.sum((uh - ex[c]) ** 2 * d.wq2[None, :])
    return np.sqrt(err2)


def test_taylor_green_spatial_velocity_error_is_third_order_for_q2q1():
    """Taylor-Hood Q2/Q1: velocity L2 error O(h^{k+2}) = O(h^3) (time error kept
    negligible by a short interval and q = 1)."""
    errs = []
    for n in (2, 4, 8):
        pb = Problem(kind="taylor_green", nu=0.05, conv=1.0, T=0.02)
        d = Discretisation(n, 1, 1, 1, pb)
        U = direct_solve(d)
        errs.append(l2_velocity_error(d, U, 0, 1))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert ratios[-1] > 6.5, (errs, ratios)


def test_taylor_green_pressure_error_is_second_order_for_q2q1():
    """Taylor-Hood Q2/Q1: pressure L2 error O(h^{k+1}) = O(h^2), with the sign
    reading Phi = -p (the discrete pressure approximates minus the strong-form
    pressure of Eq. nsfem's weak form); the Taylor-Green pressure is mean-free, like
    the discrete one."""
    errs = []
    for n in (4, 8, 16):
        pb = Problem(kind="taylor_green", nu=0.05, conv=1.0, T=0.02)
        d = Discretisation(n, 1, 1, 1, pb)
        U = direct_solve(d)
        t = d.time_nodes(0)[1]
        off = d.block(0, 1) + d.off_p
        ph = U[off:off + d.np_ ** 2][d.cell_pnodes] @ d.Vp
        ex = pb.exact_pressure(d.qpx, d.qpy, t)
        errs.append(np.sqrt(np.sum((ph + ex) ** 2 * d.wq2[None, :])))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert 3.4 < ratios[-1] < 5.5, (errs, ratios)


def test_discrete_solution_is_discretely_divergence_free():
    d = Discretisation(4, 1, 1, 2, fourier_problem())
    U = direct_solve(d)
    F = d.residual(U)
    for blk in range(d.N * d.nt):
        assert np.abs(F[blk * d.S + d.off_p:(blk + 1) * d.S]).max() < 1e-12


def _centre_stream_function(d, blk):
    """psi(1/2, y) = int_0^y u_x(1/2, s) ds of the Q2 velocity (exact per cell)."""
    nv = d.nv
    col = blk[:nv * nv].reshape(nv, nv)[:, (nv - 1) // 2]
    H = 1.0 / d.n
    ys, psi, acc = [0.0], [0.0], 0.0
    for cell in range(d.n):
        P = np.polyint(np.polyfit([0, H / 2, H], col[2 * cell:2 * cell + 3], 2))
        for s in np.linspace(0, H, 41)[1:]:
            ys.append(cell * H + s)
            psi.append(acc + np.polyval(P, s))
        acc += np.polyval(P, H)
    return np.array(ys), np.array(psi)


def test_lid_driven_cavity_data_and_steady_stokes_limit():
    """Lid data: u_x = 1 only on the open top edge.  Stokes (conv = 0) run long
    enough to be steady: the velocity is mirror-symmetric about x = 1/2 and the
    centre-line stream function has the classical Stokes-cavity minimum
    psi = -0.100076 at y = 0.7643 (the textbook value for the square cavity)."""
    pb = Problem(kind="lid", nu=1.0, conv=0.0, T=4.0)
    d = Discretisation(16, 1, 0, 4, pb)
    g = d.boundary_values()
    nv, nv2 = d.nv, d.nv ** 2
    blk0 = g[:d.S]
    top = np.zeros((nv, nv))
    top[nv - 1, 1:nv - 1] = 1.0
    assert np.array_equal(blk0[:nv2].reshape(nv, nv), top) and not blk0[nv2:].any()
    assert not d.initial_velocity().any()
    U = direct_solve(d, tol=1e-13)
    blk = U[d.block(d.N - 1, 0):d.block(d.N - 1, 0) + d.S]
    ux = blk[:nv2].reshape(nv, nv)
    uy = blk[nv2:2 * nv2].reshape(nv, nv)
    assert np.abs(ux - ux[:, ::-1]).max() < 1e-10 and np.abs(uy + uy[:, ::-1]).max() < 1e-10
    ys, psi = _centre_stream_function(d, blk)
    i = int(np.argmin(psi))
    assert abs(psi[i] + 0.100076) < 2e-4 and abs(ys[i] - 0.7643) < 0.01
    # convection breaks the mirror symmetry
    d2 = Discretisation(8, 1, 0, 2, Problem(kind="lid", nu=1.0, conv=100.0, T=0.5))
    U2 = direct_solve(d2, tol=1e-12)
    u2 = U2[d2.block(1, 0):d2.block(1, 0) + d2.nv ** 2].reshape(d2.nv, d2.nv)
    assert np.abs(u2 - u2[:, ::-1]).max() > 1e-4
