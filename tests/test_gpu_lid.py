"""The lid-driven cavity (Sec. 4) through the C ABI against the oracle: lid data
bit-exact, residual 1e-12, the whole Newton-FGMRES-WRMG solve 1e-10 with the
same FGMRES counts (Reynolds numbers 1, 10 and 100 as in the paper's tables)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fem import Discretisation
from oracle.solver import Hierarchy, Options, newton_solve
from paper_2407_13997_gb300 import inputs, wrmg
from tests.oracle_problems import oracle_problem


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("R", [1.0, 10.0, 100.0])
def test_lid_cavity_solve_matches_oracle(R):
    w = inputs.lid_cavity(n=8, k=1, q=0, N=4, R=R)
    ctx = wrmg.Context(w)
    d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
    U = ctx.vector()
    ctx.initial_guess(U)
    assert np.array_equal(U.cpu().numpy(), d.initial_guess())
    rng = np.random.default_rng(3)
    X = rng.standard_normal(d.ndofs)
    F = ctx.vector()
    ctx.residual(torch.from_numpy(X).cuda(), F)
    assert rel(F.cpu().numpy(), d.residual(X)) < 1e-12
    st = ctx.solve(U)
    ost = {}
    ref = newton_solve(Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options()), stats=ost)
    assert st["gmres"] == ost["gmres"]
    assert rel(U.cpu().numpy(), ref) < 1e-10
    ctx.close()


def test_lid_cavity_q3q2_dg1_solve_matches_oracle():
    w = inputs.lid_cavity(n=4, k=2, q=1, N=3, R=10.0)
    ctx = wrmg.Context(w)
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    ost = {}
    ref = newton_solve(Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options()), stats=ost)
    assert st["gmres"] == ost["gmres"]
    assert rel(U.cpu().numpy(), ref) < 1e-10
    ctx.close()
