"""Batching form: many solves in one lock-step batch, checked member by member
against the single-instance path (which matches the oracle): eigen-estimates to
1e-12, V-cycles and whole solves to 1e-10 relative (the batched dot products
reduce in a different order), and a member alone equal to the same member in
a mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_13997_gb300 import inputs, wrmg


def members_q2q1():
    return [inputs.fourier_small(n=8, k=1, q=0, N=3, nu=2e-2, seed=1),
            inputs.fourier_small(n=4, k=1, q=0, N=2, nu=5e-3, seed=2),
            inputs.fourier_small(n=12, k=1, q=0, N=3, nu=1e-2, seed=3, n_coarse=3),
            inputs.fourier_small(n=6, k=1, q=0, N=4, nu=3e-2, seed=4, n_coarse=3),
            inputs.fourier_small(n=16, k=1, q=0, N=2, nu=1e-3, seed=5)]


def members_q3q2():
    return [inputs.fourier_small(n=4, k=2, q=1, N=2, nu=1e-2, seed=6),
            inputs.fourier_small(n=8, k=2, q=1, N=3, nu=2e-3, seed=7)]


def rel(a, b):
    return (a - b).abs().max().item() / max(b.abs().max().item(), 1e-300)


@pytest.mark.parametrize("ws", [members_q2q1(), members_q3q2()], ids=["q2q1_dg0_mixed", "q3q2_dg1"])
def test_batched_eigen_estimates_and_vcycle_match_single_instances(ws):
    batch = wrmg.Batch(ws)
    rng = np.random.default_rng(0)
    Ws = [torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda() for w in ws]
    batch.linearise(Ws)
    bs = []
    for w in ws:
        d = w.ndofs()
        b = torch.from_numpy(rng.standard_normal(d)).cuda()
        bs.append(b)
    xs = batch.vectors()
    batch.vcycle(bs, xs)
    for m, w in enumerate(ws):
        ctx = wrmg.Context(w)
        ctx.linearise(Ws[m], eig=True)
        for l in range(1, ctx.num_levels):
            lam_s, lam_b = ctx.get_lambda(l), batch.get_lambda(m, l)
            assert abs(lam_s - lam_b) <= 1e-12 * lam_s, (m, l, lam_s, lam_b)
        x = ctx.vector()
        b = bs[m].clone()
        mask = torch.ones_like(b)
        ctx.vcycle(b, x)
        assert rel(xs[m], x) < 1e-10, m
        ctx.close()
    batch.close()


def members_solve():
    return [inputs.fourier_small(n=8, k=1, q=0, N=4, nu=2e-2, seed=1),
            inputs.fourier_small(n=4, k=1, q=0, N=3, nu=1e-2, seed=2),
            inputs.fourier_small(n=12, k=1, q=0, N=3, nu=1e-2, seed=3, n_coarse=3),
            inputs.fourier_small(n=6, k=1, q=0, N=4, nu=3e-2, seed=4, n_coarse=3),
            inputs.fourier_small(n=16, k=1, q=0, N=4, nu=5e-3, seed=5)]


def test_batched_solve_matches_single_solves_and_is_the_same_alone_and_in_the_mix():
    ws = members_solve()
    singles = []
    for w in ws:
        ctx = wrmg.Context(w)
        U = ctx.vector()
        ctx.initial_guess(U)
        st = ctx.solve(U, check=False)
        singles.append((U, st))
        ctx.close()
    batch = wrmg.Batch(ws)
    Us = batch.vectors()
    batch.initial_guess(Us)
    stats = batch.solve(Us, check=False)
    for m in range(len(ws)):
        U, st = singles[m]
        assert st["residuals"][-1] <= 1e-8 * st["residuals"][0], ("single", m, st)
        assert stats[m]["residuals"][-1] <= 1e-8 * stats[m]["residuals"][0], ("batched", m, stats[m], st)
        assert stats[m]["newton_its"] == st["newton_its"], (m, stats[m], st)
        assert rel(Us[m], U) < 1e-10, m
    # member 2 alone in a batch of one
    alone = wrmg.Batch([ws[2]])
    Ua = alone.vectors()
    alone.initial_guess(Ua)
    alone.solve(Ua)
    assert rel(Ua[0], Us[2]) < 1e-10
    alone.close()
    batch.close()


def test_graph_replay_equals_eager_cycles_bitwise():
    """The batched V-cycle captured as one CUDA graph (re-captured when the active
    set changes) gives bitwise the eager cycle's result, and its kernels are counted
    once per replay."""
    ws = members_q2q1()
    rng = np.random.default_rng(5)
    Ws = [torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda() for w in ws]
    bs = [torch.from_numpy(rng.standard_normal(w.ndofs())).cuda() for w in ws]
    out = []
    for graphs in (True, False):
        batch = wrmg.Batch(ws)
        batch.set_graphs(graphs)
        batch.linearise(Ws)
        xs = batch.vectors()
        for _ in range(3):                       # capture, then replays
            batch.vcycle(bs, xs)
        torch.cuda.synchronize()
        n0 = wrmg.launch_count()
        batch.vcycle(bs, xs)
        torch.cuda.synchronize()
        per_cycle = wrmg.launch_count() - n0
        Us = batch.vectors()
        batch.initial_guess(Us)
        st = batch.solve(Us, check=False)
        out.append((xs, per_cycle, Us, [s["gmres"] for s in st]))
        batch.close()
    (xg, ng, Ug, gg), (xe, ne, Ue, ge) = out
    assert all(torch.equal(a, b) for a, b in zip(xg, xe))
    assert ng == ne > 10
    assert gg == ge
    assert all(torch.equal(a, b) for a, b in zip(Ug, Ue))


@pytest.mark.parametrize("tile", [2, 3, 4])
def test_batched_apply_tiles_match_single_instances(tile):
    ws = members_q2q1()
    rng = np.random.default_rng(8)
    Ws = [torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda() for w in ws]
    batch = wrmg.Batch(ws, wrmg.default_options(apply_tile=tile))
    batch.linearise(Ws)
    bs = [torch.from_numpy(rng.standard_normal(w.ndofs())).cuda() for w in ws]
    xs = batch.vectors()
    batch.vcycle(bs, xs)
    for m, w in enumerate(ws):
        ctx = wrmg.Context(w, wrmg.default_options(apply_tile=tile, time_parallel=0))
        ctx.linearise(Ws[m], eig=True)
        x = ctx.vector()
        ctx.vcycle(bs[m].clone(), x)
        assert rel(xs[m], x) < 1e-10, m
        ctx.close()
    batch.close()
