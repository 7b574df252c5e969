"""The heat equation (Def. heat, Sec. 5) through the C ABI against the oracle:
patch index tables bit-exact, operator and transfers 1e-12/1e-13, smoother,
coarse solve, eigen-estimates and V-cycle 1e-10, the FGMRES-WRMG solve with the
same iteration count and 1e-10 on the solution, and the timestepping comparator
equal to the all-at-once solve; Q_k (k = 1..3) x DG(q) (q = 0..3)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.heat import (HeatCoarseSolver, HeatDiscretisation, HeatHierarchy, HeatProblem, HeatSmoother,
                         heat_patch_dofs, heat_prolongation, heat_solve)
from oracle.solver import Options
from paper_2407_13997_gb300 import inputs, wrmg

CASES = [inputs.heat(n=8, k=1, q=0, N=5), inputs.heat(n=8, k=2, q=1, N=4), inputs.heat(n=4, k=3, q=1, N=3),
         inputs.heat(n=8, k=3, q=0, N=3, eigen=True),
         # DG(2) and DG(3) in time (Sec. 5's temporal degrees); k = q = 3 coarsens to 1x1,
         # k = 3, q = 2 takes the largest 2x2 coarse block (147 x 147)
         inputs.heat(n=8, k=1, q=2, N=3), inputs.heat(n=4, k=2, q=3, N=3), inputs.heat(n=4, k=3, q=3, N=2),
         inputs.heat(n=4, k=3, q=2, N=2)]
IDS = [w.name + ("_eig" if w.kind == inputs.KIND_HEAT_EIGEN else "") for w in CASES]


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle_hier(w, opts=None):
    pb = HeatProblem(nu=w.nu, T=w.T, u0="cos" if w.kind == inputs.KIND_HEAT_EIGEN else "paper")
    return HeatHierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, pb, opts)


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def setup(request):
    w = request.param
    ctx = wrmg.Context(w)
    hier = oracle_hier(w)
    yield w, ctx, hier
    ctx.close()


def test_patch_tables_operator_and_residual(setup):
    w, ctx, hier = setup
    assert ctx.num_levels == len(hier.discs)
    rng = np.random.default_rng(1)
    for l, d in enumerate(hier.discs):
        assert ctx.ndofs(l) == d.ndofs
        if l >= 1:
            for patch in range((d.n + 1) ** 2):
                assert np.array_equal(ctx.patch_dofs(l, patch, d.N - 1), heat_patch_dofs(d, patch, d.N - 1))
        x = rng.standard_normal(d.ndofs)
        y = ctx.vector(l)
        ctx.apply_jacobian(l, cuda(x), y)
        assert rel(y.cpu().numpy(), hier.J[l] @ x) < 1e-12, l
    U = rng.standard_normal(hier.fine.ndofs)
    F = ctx.vector()
    ctx.residual(cuda(U), F)
    assert rel(F.cpu().numpy(), hier.fine.residual(U)) < 1e-12


def test_transfers_smoother_coarse_solve_and_vcycle(setup):
    w, ctx, hier = setup
    rng = np.random.default_rng(2)
    ctx.linearise(ctx.vector(), eig=True)
    for l in range(1, len(hier.discs)):
        P = hier.P[l]
        xf = rng.standard_normal(hier.discs[l].ndofs)
        xc = rng.standard_normal(hier.discs[l - 1].ndofs)
        oc = ctx.vector(l - 1)
        ctx.restrict(l, cuda(xf), oc)
        assert rel(oc.cpu().numpy(), P.T @ xf) < 1e-13
        of = cuda(xf.copy())
        ctx.prolong_add(l, cuda(xc), of)
        assert rel(of.cpu().numpy(), xf + P @ xc) < 1e-13
        r = rng.standard_normal(hier.discs[l].ndofs)
        y = ctx.vector(l)
        ctx.patch_apply(l, cuda(r), y)
        assert rel(y.cpu().numpy(), hier.smoothers[l].apply(r)) < 1e-10, l
        assert abs(ctx.get_lambda(l) - hier.lam[l]) < 1e-10 * hier.lam[l]
    b0 = rng.standard_normal(hier.discs[0].ndofs)
    x0 = ctx.vector(0)
    ctx.coarse_solve(cuda(b0), x0)
    assert rel(x0.cpu().numpy(), hier.coarse.solve(b0)) < 1e-10
    b = rng.standard_normal(hier.fine.ndofs)
    x = ctx.vector()
    ctx.vcycle(cuda(b), x)
    assert rel(x.cpu().numpy(), hier.vcycle(b)) < 1e-10


def heat_options(rtol=1e-6):
    return wrmg.default_options(newton_maxit=1, ew=0, eta_fixed=rtol, newton_rtol=rtol)


@pytest.mark.parametrize("w", CASES, ids=IDS)
def test_fgmres_wrmg_solve_matches_oracle(w):
    ctx = wrmg.Context(w, heat_options())
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    Uref, its = heat_solve(oracle_hier(w), rtol=1e-6, atol=0.0)
    assert st["gmres"] == [its]
    assert rel(U.cpu().numpy(), Uref) < 1e-10
    ctx.close()


def test_heat_timestepping_equals_all_at_once():
    w = inputs.heat(n=8, k=2, q=1, N=4)
    tight = heat_options(1e-13)
    c1 = wrmg.Context(dataclasses.replace(w, N=1, T=w.T / w.N), tight)
    Ut = torch.zeros(w.ndofs(), dtype=torch.float64, device="cuda")
    c1.solve_timestepping(Ut, w.N, check=False)
    c2 = wrmg.Context(w, tight)
    Ua = c2.vector()
    c2.initial_guess(Ua)
    c2.solve(Ua, check=False)
    assert rel(Ut.cpu().numpy(), Ua.cpu().numpy()) < 1e-9
    c1.close()
    c2.close()
