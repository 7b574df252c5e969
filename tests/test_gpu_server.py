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
