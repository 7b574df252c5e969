"""Precision form: FP32 stored patch factors and FP32 smoother arithmetic, with the
residual, FGMRES (Arnoldi, Givens, least squares) and the coarse solve in FP64.

The smoother itself is only FP32-accurate, so it is compared with the FP64 oracle
at 2e-5 relative (FP32 rounding of inverses with condition numbers up to ~1e2);
whole solves are run to a tight residual (1e-11) so that both the FP32-smoother
solution and the FP64 oracle solution sit well inside the 1e-8 bound on the
final solution that the precision form must meet.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fem import Discretisation
from oracle.patches import PatchSmoother
from oracle.solver import Hierarchy, Options, newton_solve
from oracle.transfer import injection
from paper_2407_13997_gb300 import inputs, wrmg
from tests.oracle_problems import oracle_problem


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec,lo,hi", [("fp32", 1e-12, 2e-5), ("bf16", 1e-5, 0.25)])
@pytest.mark.parametrize("w", [inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02),
                               inputs.fourier_small(n=4, k=2, q=1, N=2, nu=0.01)], ids=["q2q1_dg0", "q3q2_dg1"])
def test_reduced_precision_smoother_close_to_fp64_oracle(w, prec, lo, hi):
    """FP32: FP32-accurate; BF16 factors (8-bit mantissa) with FP32 arithmetic:
    BF16-accurate (2^-9 rounding per entry, compounded through the factored blocks and
    amplified by their conditioning: a few per cent)."""
    ctx = wrmg.Context(w, wrmg.default_options(precision={"fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16}[prec]))
    d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
    rng = np.random.default_rng(5)
    W = 0.5 * rng.standard_normal(d.ndofs)
    mask = d.dirichlet_mask()
    W[mask] = d.boundary_values()[mask]
    ctx.linearise(torch.from_numpy(W).cuda(), eig=False)
    r = rng.standard_normal(d.ndofs)
    y = ctx.vector()
    ctx.patch_apply(ctx.fine, torch.from_numpy(r).cuda(), y)
    ref = PatchSmoother(d, d.jacobian(W)).apply(r)
    err = rel(y.cpu().numpy(), ref)
    assert lo < err < hi, err   # genuinely reduced precision, and as accurate as that precision allows
    ctx.close()


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec,lo,hi", [("fp32", 1e-12, 2e-5), ("bf16", 1e-5, 0.25)])
@pytest.mark.parametrize("w", [inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02),
                               inputs.fourier_small(n=8, k=1, q=1, N=2, nu=0.02)], ids=["q2q1_dg0", "q2q1_dg1"])
def test_reduced_precision_every_tile_close_to_fp64_oracle(w, prec, lo, hi, tile):
    """Every apply tile on every smoothed level of Q2/Q1, in FP32 and BF16.  The BF16
    Q2/Q1 blocks are stored by column octets (written by the warp factor kernel for DG(0)
    and by the CTA factor kernel for DG(1)); the warp tiles read them one 16-byte word per
    row and octet and the CTA tiles one octet per thread, the last three columns column by
    column.  A misplaced entry would put the smoother far outside the precision's band."""
    from tests.test_gpu_parity import Setup
    p = {"fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16}[prec]
    s = Setup(w, seed=3, options=wrmg.default_options(precision=p, apply_tile=tile, time_parallel=0))
    s.ctx.linearise(torch.from_numpy(s.W[-1]).cuda(), eig=False)
    for l in range(1, len(s.discs)):
        d = s.discs[l]
        assert s.ctx.apply_tile(l) == tile
        r = s.rng.standard_normal(d.ndofs)
        y = s.ctx.vector(l)
        s.ctx.patch_apply(l, torch.from_numpy(r).cuda(), y)
        err = rel(y.cpu().numpy(), PatchSmoother(d, d.jacobian(s.W[l])).apply(r))
        assert lo < err < hi, (l, err)
    s.ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("w", [inputs.taylor_green_8x8(), inputs.fourier_small(n=8, k=2, q=1, N=4, nu=1e-2)],
                         ids=["tg_q2q1_dg0_n8_N8", "fourier_q3q2_dg1_n8_N4"])
def test_reduced_precision_solve_meets_1e8_against_fp64_oracle(w, prec):
    opts = wrmg.default_options(precision={"fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16}[prec], newton_rtol=1e-11)
    ctx = wrmg.Context(w, opts)
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    hier = Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options(newton_rtol=1e-11))
    ref = newton_solve(hier)
    err = rel(U.cpu().numpy(), ref)
    assert err <= 1e-8, (err, st)
    ctx.close()


@pytest.mark.parametrize("w", [inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02),
                               inputs.fourier_small(n=8, k=2, q=1, N=2, nu=0.01)], ids=["q2q1_dg0", "q3q2_dg1"])
def test_fp32_form_vcycle_close_to_fp64_oracle(w):
    """In the FP32 form every operator inside the V-cycle (the patch smoother and the
    Jacobian actions of the Chebyshev residuals and of the restricted residual) is
    single precision; the cycle stays FP32-accurate against the FP64 oracle's."""
    ctx = wrmg.Context(w, wrmg.default_options(precision=wrmg.WR_FP32))
    hier = Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options())
    rng = np.random.default_rng(9)
    d = hier.fine
    W = 0.5 * rng.standard_normal(d.ndofs)
    mask = d.dirichlet_mask()
    W[mask] = d.boundary_values()[mask]
    hier.linearise(W)
    ctx.linearise(torch.from_numpy(W).cuda(), eig=False)
    for l in range(1, len(hier.levels)):
        ctx.set_lambda(l, hier.levels[l].lam)
    b = rng.standard_normal(d.ndofs) * hier.levels[-1].free
    x = ctx.vector()
    ctx.vcycle(torch.from_numpy(b).cuda(), x)
    err = rel(x.cpu().numpy(), hier.vcycle(b))
    assert 1e-12 < err < 1e-4, err
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
def test_bulk_copy_warp_tile_equals_the_warp_tile_bitwise(prec):
    """Tile 4 (a warp per patch, each slab's block bulk-copied into shared memory two
    slabs ahead) performs tile 3's arithmetic in tile 3's order: the smoother outputs
    agree bit for bit on every level, for Q2/Q1 DG(0) in every factor precision, with
    a slab count that exercises both buffers and the copies issued two slabs ahead."""
    w = inputs.fourier_small(n=16, k=1, q=0, N=7, nu=0.02)
    p = {"fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16, "fp64": wrmg.WR_FP64}[prec]
    rng = np.random.default_rng(11)
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    outs = {}
    for tile in (3, 4):
        ctx = wrmg.Context(w, wrmg.default_options(precision=p, apply_tile=tile, time_parallel=0))
        ctx.linearise(W, eig=False)
        rng = np.random.default_rng(11)
        res = []
        for l in range(1, ctx.num_levels):
            assert ctx.apply_tile(l) == tile
            r = torch.from_numpy(rng.standard_normal(ctx.ndofs(l))).cuda()
            y = ctx.vector(l)
            ctx.patch_apply(l, r, y)
            res.append(y.cpu().numpy())
        outs[tile] = res
        ctx.close()
    for a, b in zip(outs[3], outs[4]):
        assert np.array_equal(a, b)
