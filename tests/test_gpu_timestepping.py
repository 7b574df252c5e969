"""The timestepping comparator and the time offset / initial state it rests on,
through the C ABI, against the oracle.

A one-slab context moved along the time axis solves slab after slab with the
previous end state as the slab-0 initial data (Sec. 5's timestepping analogue
of WRMG).  Residuals with a start time and a given initial state match the
oracle to 1e-12; the GPU timestepping loop matches the oracle's to 1e-10 with
the same FGMRES counts; and because the space-time system is causal, the
timestepped solution equals the all-at-once WRMG solution to the solver
tolerance (both run to 1e-12 here).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fem import Discretisation
from oracle.solver import Hierarchy, Options, newton_solve, timestepping_solve
from paper_2407_13997_gb300 import inputs, wrmg
from tests.oracle_problems import oracle_problem


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def tg(n=4, k=1, q=1, N=3, T=0.6, t0=0.0):
    return inputs.Workload(f"tg_k{k}_q{q}_n{n}_N{N}", n, 2, k, q, N, T, 0.05, 1.0, inputs.KIND_TAYLOR_GREEN, t0=t0)


def poly(n=4, k=2, q=1, N=3, T=0.6, t0=0.0):
    return inputs.Workload(f"poly_k{k}_q{q}_n{n}_N{N}", n, 2, k, q, N, T, 0.05, 1.0, inputs.KIND_POLY, t0=t0)


@pytest.mark.parametrize("w", [tg(N=2, t0=0.3), poly(N=2, t0=0.45)], ids=["tg", "poly"])
def test_residual_with_start_time_and_initial_state_matches_oracle(w):
    ctx = wrmg.Context(w)
    d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
    rng = np.random.default_rng(1)
    U = rng.standard_normal(d.ndofs)
    F = ctx.vector()
    ctx.residual(torch.from_numpy(U).cuda(), F)
    assert rel(F.cpu().numpy(), d.residual(U)) < 1e-12
    G = ctx.vector()
    ctx.initial_guess(G)
    assert rel(G.cpu().numpy(), d.initial_guess()) < 1e-14
    u0 = rng.standard_normal(d.S)
    ctx.set_initial_state(torch.from_numpy(u0).cuda())
    ctx.residual(torch.from_numpy(U).cuda(), F)
    d.initial_state = u0
    assert rel(F.cpu().numpy(), d.residual(U)) < 1e-12
    ctx.set_initial_state(None)
    d.initial_state = None
    ctx.residual(torch.from_numpy(U).cuda(), F)
    assert rel(F.cpu().numpy(), d.residual(U)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("w", [tg(), poly(), tg(n=8, q=0, N=4, T=0.8)], ids=["tg_q1", "poly_q3q2", "tg_q0"])
def test_timestepping_matches_oracle_and_the_all_at_once_solution(w):
    one = dataclasses.replace(w, N=1, T=w.T / w.N)
    ctx = wrmg.Context(one)
    U = torch.zeros(w.ndofs(), dtype=torch.float64, device="cuda")
    st = ctx.solve_timestepping(U, w.N)
    ost = {}
    ref = timestepping_solve(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options(), stats=ost)
    assert rel(U.cpu().numpy(), ref) < 1e-10
    assert st["gmres_per_step"] == [sum(s["gmres"]) for s in ost["steps"]]
    ctx.close()
    # causality: the all-at-once solution is the timestepped one (both to 1e-12)
    tight = wrmg.default_options(newton_rtol=1e-12, ew=0, eta_fixed=1e-12)
    c1 = wrmg.Context(one, tight)
    Ut = torch.zeros(w.ndofs(), dtype=torch.float64, device="cuda")
    c1.solve_timestepping(Ut, w.N)
    c2 = wrmg.Context(w, tight)
    Ua = c2.vector()
    c2.initial_guess(Ua)
    c2.solve(Ua)
    assert rel(Ut.cpu().numpy(), Ua.cpu().numpy()) < 1e-9
    c1.close()
    c2.close()
