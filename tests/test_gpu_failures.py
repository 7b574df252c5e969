"""Failure detection without a GPU fault: every failure here is made on the host
(an allocation that fails, a NaN in an input, a cancelled request) or is a
bounded device wait that runs out on a barrier nothing completes; the context
stays usable after each."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_13997_gb300 import inputs, wrmg

W = inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02)


def test_bounded_wait_gives_up_and_reports():
    timed_out, ms = wrmg.selftest_bounded_wait(torch.cuda.current_stream().cuda_stream)
    assert timed_out
    assert 1500.0 < ms < 10000.0
    # the device is still usable
    ctx = wrmg.Context(W)
    U = ctx.vector()
    ctx.initial_guess(U)
    assert ctx.solve(U)["status"] == wrmg.WR_OK
    ctx.close()


def test_injected_allocation_failure_is_reported_and_recovered():
    wrmg.inject_alloc_failure(5)
    with pytest.raises(wrmg.WrmgError) as e:
        wrmg.Context(W)
    assert e.value.code == wrmg.WR_ERR_NOMEM and "injected" in str(e.value)
    ctx = wrmg.Context(W)            # the injection fired once; creation works again
    ctx.close()
    wrmg.inject_alloc_failure(3)     # inside the server: the request fails, the server goes on
    sv = wrmg.Server(1 << 30, 2)
    t1 = sv.submit(W)
    r1 = sv.poll(t1)
    wrmg.inject_alloc_failure(0)
    t2 = sv.submit(W)
    r2 = sv.poll(t2)
    sv.close()
    assert r1[0] == wrmg.WR_ERR_NOMEM and r2[0] == wrmg.WR_OK


def test_nan_in_the_iterate_is_detected():
    ctx = wrmg.Context(W)
    U = ctx.vector()
    ctx.initial_guess(U)
    U[ctx.ndofs() // 2] = float("nan")
    st = ctx.solve(U, check=False)
    assert st["status"] == wrmg.WR_ERR_NAN
    U2 = ctx.vector()
    ctx.initial_guess(U2)
    assert ctx.solve(U2)["status"] == wrmg.WR_OK
    ctx.close()


def test_cancelled_requests_queued_and_running():
    big = inputs.fourier_small(n=32, k=2, q=1, N=8, nu=0.02)
    sv = wrmg.Server(64 << 30, 1)
    t_run = sv.submit(big)          # admitted at once (one slot)
    t_wait = sv.submit(W)           # queued behind it
    t_keep = sv.submit(W)
    sv.cancel(t_wait)
    sv.cancel(t_run)
    r_run, r_wait, r_keep = sv.poll(t_run), sv.poll(t_wait), sv.poll(t_keep)
    sv.close()
    assert r_wait[0] == wrmg.WR_ERR_CANCELLED
    assert r_run[0] in (wrmg.WR_ERR_CANCELLED, wrmg.WR_OK)   # it may finish before the flag is seen
    assert r_keep[0] == wrmg.WR_OK


def test_newton_safeguards_match_the_oracle():
    """Divergence and FGMRES-stagnation safeguards stop Newton where the oracle's do."""
    from oracle.fem import Problem
    from oracle.solver import Hierarchy, Options, newton_solve
    w = inputs.fourier_small(n=4, k=1, q=0, N=2, nu=0.02)
    from tests.oracle_problems import oracle_problem
    for gpu_opts, ora_opts in [(dict(newton_divtol=0.5), dict(newton_divtol=0.5)),
                               (dict(gmres_maxit=1, newton_stall=2), dict(gmres_maxit=1, newton_stall=2))]:
        ctx = wrmg.Context(w, wrmg.default_options(**gpu_opts))
        U = ctx.vector()
        ctx.initial_guess(U)
        st = ctx.solve(U, check=False)
        ost = {}
        newton_solve(Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options(**ora_opts)),
                     stats=ost)
        assert st["status"] == wrmg.WR_ERR_NOT_CONVERGED
        assert st["gmres"] == ost["gmres"]
        ctx.close()
