"""Parity at the full 64x64 Q3/Q2 DG(1), 64-slab workload (11,665,792 DoFs) in the
launch configuration bench.py times, on outputs the oracle can compute one slab
or one patch at a time, plus properties that hold at any size.

Tolerances: residual and Jacobian rows 1e-12 relative (same FP64 quadrature,
different summation order); transfers 1e-13; smoother response 1e-10 (inverses
of patch blocks amplify rounding by their condition number).
"""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fem import Discretisation
from oracle.patches import patch_dofs
from oracle.transfer import spatial_prolongation
from paper_2407_13997_gb300 import inputs, wrmg
from tests.oracle_problems import oracle_problem


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def big():
    w = inputs.fourier_64x64_q3q2_dg1(0)
    ctx = wrmg.Context(w)
    W = inputs.forcing_shaped_iterate(w)
    Wd = torch.from_numpy(W).cuda()
    ctx.linearise(Wd, eig=True)
    d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
    yield w, ctx, W, Wd, d
    ctx.close()


def slab(d, v, n):
    return v[d.block(n, 0):d.block(n + 1, 0)]


def test_residual_rows_match_oracle(big):
    w, ctx, W, Wd, d = big
    F = ctx.vector()
    ctx.residual(Wd, F)
    F = F.cpu().numpy()
    for n in (0, 1, w.N - 1):
        assert rel(slab(d, F, n), d.residual_slab(W, n)) < 1e-12, n


def test_jacobian_rows_match_oracle(big):
    w, ctx, W, Wd, d = big
    x = np.random.default_rng(3).standard_normal(d.ndofs)
    y = ctx.vector()
    ctx.apply_jacobian(ctx.fine, torch.from_numpy(x).cuda(), y)
    y = y.cpu().numpy()
    for n in (0, 1, w.N - 1):
        D, L = d.jacobian_slab(W, n)
        ref = D @ slab(d, x, n) + (L @ slab(d, x, n - 1) if n > 0 else 0.0)
        assert rel(slab(d, y, n), ref) < 1e-12, n


def test_transfers_match_oracle(big):
    w, ctx, W, Wd, d = big
    L = ctx.fine
    dc = Discretisation(w.n_fine // 2, w.k, w.q, w.N, oracle_problem(w))
    Ph = spatial_prolongation(d, dc)
    rng = np.random.default_rng(4)
    xf = rng.standard_normal(d.ndofs)
    xc = rng.standard_normal(dc.ndofs)
    oc = ctx.vector(L - 1)
    ctx.restrict(L, torch.from_numpy(xf).cuda(), oc)
    of = torch.from_numpy(xf.copy()).cuda()
    ctx.prolong_add(L, torch.from_numpy(xc).cuda(), of)
    oc, of = oc.cpu().numpy(), of.cpu().numpy()
    for blk in (0, 37, d.N * d.nt - 1):
        f = slice(blk * d.S, (blk + 1) * d.S)
        c = slice(blk * dc.S, (blk + 1) * dc.S)
        assert rel(oc[c], Ph.T @ xf[f]) < 1e-13
        assert rel(of[f], xf[f] + Ph @ xc[c]) < 1e-13


@pytest.mark.parametrize("which", ["velocity_vertex", "pressure_edge"])
def test_smoother_response_to_a_unit_vector_matches_oracle(big, which):
    """M^{-1} e_d involves only the patches that contain DoF d and, by the forward
    substitution, only slabs >= slab(d); the oracle recomputes those patches'
    waveform solves on two slabs from their principal submatrices."""
    w, ctx, W, Wd, d = big
    n0 = 2
    if which == "velocity_vertex":
        dof = d.block(n0, 0) + d.vel_index(0, 96, 96)     # vertex node of 9 patches
        I0, J0 = 32, 32
        cand = [(I, J) for J in (J0 - 1, J0, J0 + 1) for I in (I0 - 1, I0, I0 + 1)]
    else:
        dof = d.block(n0, 1) + d.pres_index(63, 64)       # mid-edge pressure node of 2 patches
        cand = [(31, 32), (32, 32)]
    r = np.zeros(d.ndofs)
    r[dof] = 1.0
    y = ctx.vector()
    ctx.patch_apply(ctx.fine, torch.from_numpy(r).cuda(), y)
    y = y.cpu().numpy()
    assert np.all(y[:d.block(n0, 0)] == 0.0)            # causality of the forward substitution
    blocks = {n: d.jacobian_slab(W, n) for n in (n0, n0 + 1)}
    ref = np.zeros(d.ndofs)
    touched = np.zeros(d.ndofs, dtype=bool)
    for I, J in cand:
        p = J * (d.n + 1) + I
        ix0, ix1 = patch_dofs(d, p, n0), patch_dofs(d, p, n0 + 1)
        assert dof in ix0
        l0, l1 = ix0 - d.block(n0, 0), ix1 - d.block(n0 + 1, 0)
        D0, _ = blocks[n0]
        D1, L1 = blocks[n0 + 1]
        y0 = sla.solve(D0[l0][:, l0].toarray(), r[ix0])
        y1 = sla.solve(D1[l1][:, l1].toarray(), r[ix1] - L1[l1][:, l0].toarray() @ y0)
        ref[ix0] += y0
        ref[ix1] += y1
        touched[ix0] = touched[ix1] = True
    win = slice(d.block(n0, 0), d.block(n0 + 2, 0))
    assert rel(y[win], ref[win]) < 1e-10
    assert np.all(y[win][~touched[win]] == 0.0)         # nothing outside the patches that hold d


def test_vcycle_is_linear_reproducible_and_contracting(big):
    w, ctx, W, Wd, d = big
    F = ctx.vector()
    ctx.residual(Wd, F)
    b1 = -F
    mask = torch.from_numpy(~d.dirichlet_mask()).cuda()
    b2 = torch.from_numpy(np.random.default_rng(5).standard_normal(d.ndofs)).cuda() * mask
    v1, v1b, v2, v12 = ctx.vector(), ctx.vector(), ctx.vector(), ctx.vector()
    ctx.vcycle(b1, v1)
    ctx.vcycle(b1, v1b)
    ctx.vcycle(b2, v2)
    ctx.vcycle(b1 + 2.0 * b2, v12)
    assert torch.equal(v1, v1b)                          # deterministic: bitwise reproducible
    lin = (v12 - v1 - 2.0 * v2).abs().max().item() / v12.abs().max().item()
    assert lin < 1e-11
    Jv = ctx.vector()
    ctx.apply_jacobian(ctx.fine, v1, Jv)
    ratio = (b1 - Jv).norm().item() / b1.norm().item()
    assert ratio < 0.5, ratio
    dm = torch.from_numpy(d.dirichlet_mask()).cuda()
    assert v1[dm].abs().max().item() == 0.0


def test_newton_solve_converges_at_full_size(big):
    """The whole Newton-FGMRES-WRMG solve of the 11.7M-DoF workload reaches 1e-8."""
    w, ctx, W, Wd, d = big
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    assert st["residuals"][-1] <= 1e-8 * st["residuals"][0], st
    assert st["newton_its"] <= 8 and max(st["gmres"]) <= 40, st
    print("full-size solve:", st)
