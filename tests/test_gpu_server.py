"""The serving form (wr_server_*) and the allocation estimator, through the C ABI.

Each request of a server runs on its own stream and context with the same
deterministic kernels as a solve alone, so a solve's result must not depend on
what else is in flight: every served result is compared bit for bit with a
Context solve of that problem alone.  Admission must respect the memory budget
and the in-flight cap, and a request larger than the whole budget is refused
with WR_ERR_NOMEM without disturbing the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_13997_gb300 import inputs, wrmg

MIX = [
    inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02),
    inputs.fourier_small(n=4, k=2, q=1, N=2, nu=0.01),
    inputs.taylor_green_8x8(),
    inputs.poly_small(n=4, k=2, q=1, N=2),
    inputs.fourier_small(n=12, k=1, q=1, N=2, nu=0.02, n_coarse=3),
    inputs.fourier_small(n=16, k=1, q=0, N=4, nu=0.02),
]


def alone(w, options=None):
    ctx = wrmg.Context(w, options)
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    torch.cuda.synchronize()
    ctx.close()
    return U.cpu().numpy(), st


def request_bytes(w, options=None):
    return wrmg.estimate_bytes(w, options) + 8 * w.ndofs()


@pytest.mark.parametrize("prec", [wrmg.WR_FP64, wrmg.WR_FP32, wrmg.WR_BF16], ids=["fp64", "fp32", "bf16"])
def test_estimate_equals_allocated_bytes(prec):
    o = wrmg.default_options(precision=prec)
    for w in MIX[:3] + [inputs.fourier_64x64_q3q2_dg1()]:
        if w.n_fine == 64:
            w.N = 4          # same per-slab layout, smaller allocation
        ctx = wrmg.Context(w, o)
        assert ctx.device_bytes() == wrmg.estimate_bytes(w, o), w.name
        ctx.close()


def test_served_results_equal_solves_alone():
    refs = [alone(w) for w in MIX]
    sv = wrmg.Server(mem_budget_bytes=4 << 30, max_inflight=3)
    tickets = [sv.submit(w) for w in MIX]
    # the same first problem again, with its Dirichlet start given explicitly
    ctx = wrmg.Context(MIX[0])
    U0 = ctx.vector()
    ctx.initial_guess(U0)
    tickets.append(sv.submit(MIX[0], U0=U0.cpu().numpy()))
    ctx.close()
    out = [sv.poll(t) for t in tickets]
    stats = sv.stats()
    sv.close()
    for (rc, U, st, lat), (Uref, stref), w in zip(out, refs + [refs[0]], MIX + [MIX[0]]):
        assert rc == wrmg.WR_OK, w.name
        assert np.array_equal(U, Uref), w.name
        assert st["gmres"] == stref["gmres"], w.name
        assert lat > 0.0
    assert 1 <= stats["peak_inflight"] <= 3
    assert stats["peak_bytes"] <= 4 << 30


def test_budget_admission_and_refusal():
    sizes = [request_bytes(w) for w in MIX]
    budget = max(sizes) + min(sizes)            # the largest plus the smallest fit together, no more
    big = inputs.fourier_small(n=32, k=2, q=1, N=8, nu=0.02)
    assert request_bytes(big) > budget
    sv = wrmg.Server(mem_budget_bytes=budget, max_inflight=8)
    tickets = [sv.submit(w) for w in MIX[:3]] + [sv.submit(big)] + [sv.submit(w) for w in MIX[3:]]
    out = [sv.poll(t) for t in tickets]
    stats = sv.stats()
    sv.close()
    codes = [o[0] for o in out]
    assert codes[3] == wrmg.WR_ERR_NOMEM
    assert all(c == wrmg.WR_OK for i, c in enumerate(codes) if i != 3)
    assert stats["peak_bytes"] <= budget
    assert stats["peak_inflight"] >= 1


def test_poll_without_wait_and_unknown_ticket():
    sv = wrmg.Server(mem_budget_bytes=1 << 30, max_inflight=1)
    t = sv.submit(MIX[0])
    res = None
    for _ in range(200000):
        res = sv.poll(t, wait=False)
        if res is not None:
            break
    if res is None:
        res = sv.poll(t, wait=True)
    assert res[0] == wrmg.WR_OK
    sv.close()


def test_batched_server_results_equal_solves_alone_and_cohorts_form():
    """Per-cycle (continuous) batching: with one slot, requests queued while a
    cohort runs are solved together in the next cohort (one lock-step batch); every
    result equals the solve of that problem alone within the parity tolerance and
    takes the same FGMRES iterations, whatever cohort it landed in."""
    mix = [w for w in MIX if w.q <= 1]
    refs = [alone(w) for w in mix]
    sv = wrmg.Server(mem_budget_bytes=8 << 30, max_inflight=1, batch_members=8)
    tickets = [sv.submit(w) for w in mix]
    ctx = wrmg.Context(mix[0])
    U0 = ctx.vector()
    ctx.initial_guess(U0)
    tickets.append(sv.submit(mix[0], U0=U0.cpu().numpy()))
    ctx.close()
    out = [sv.poll(t) for t in tickets]
    stats = sv.stats()
    sv.close()
    for (rc, U, st, lat), (Uref, stref), w in zip(out, refs + [refs[0]], mix + [mix[0]]):
        assert rc == wrmg.WR_OK, w.name
        assert np.abs(U - Uref).max() <= 1e-10 * np.abs(Uref).max(), w.name
        assert st["gmres"] == stref["gmres"], w.name
        assert lat > 0.0
    assert stats["peak_inflight"] == 1
    assert stats["peak_cohort"] >= 2
    assert stats["peak_bytes"] <= 8 << 30


def test_batched_server_is_the_same_alone_and_in_the_mix():
    """A request served in a cohort of eight and served alone give the same result
    within the parity tolerance."""
    w = inputs.fourier_small(n=8, k=1, q=0, N=4, nu=0.02, seed=7)
    others = [inputs.fourier_small(n=n, k=1, q=0, N=N, nu=nu, seed=s)
              for n, N, nu, s in [(8, 3, 0.05, 1), (16, 2, 0.02, 2), (4, 4, 0.01, 3), (8, 8, 0.03, 4),
                                  (16, 4, 0.02, 5), (4, 2, 0.05, 6), (8, 2, 0.02, 8)]]
    sv = wrmg.Server(mem_budget_bytes=8 << 30, max_inflight=1, batch_members=1 + len(others))
    t_alone = sv.submit(w)
    rc, U_alone, st_alone, _ = sv.poll(t_alone)
    tickets = [sv.submit(o) for o in others[:3]] + [sv.submit(w)] + [sv.submit(o) for o in others[3:]]
    out = [sv.poll(t) for t in tickets]
    stats = sv.stats()
    sv.close()
    assert rc == wrmg.WR_OK and all(o[0] == wrmg.WR_OK for o in out)
    rc2, U_mix, st_mix, _ = out[3]
    assert np.abs(U_mix - U_alone).max() <= 1e-10 * np.abs(U_alone).max()
    assert st_mix["gmres"] == st_alone["gmres"]
    assert stats["peak_cohort"] >= 2


def test_batched_server_budget_refusal_and_cancel():
    sizes = [request_bytes(w) for w in MIX]
    budget = max(sizes) + min(sizes)
    big = inputs.fourier_small(n=32, k=2, q=1, N=8, nu=0.02)
    sv = wrmg.Server(mem_budget_bytes=budget, max_inflight=2, batch_members=4)
    tickets = [sv.submit(w) for w in MIX[:3]] + [sv.submit(big)] + [sv.submit(w) for w in MIX[3:]]
    last = sv.submit(MIX[0])
    sv.cancel(last)
    out = [sv.poll(t) for t in tickets]
    rc_last = sv.poll(last)[0]
    stats = sv.stats()
    sv.close()
    codes = [o[0] for o in out]
    assert codes[3] == wrmg.WR_ERR_NOMEM
    assert all(c == wrmg.WR_OK for i, c in enumerate(codes) if i != 3)
    assert rc_last in (wrmg.WR_OK, wrmg.WR_ERR_CANCELLED)
    assert stats["peak_bytes"] <= budget
