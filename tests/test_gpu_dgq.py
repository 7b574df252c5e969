"""Navier-Stokes with the higher temporal orders DG(2) and DG(3) (Sec. 2's DG(q) in
time; the paper's higher-order experiments), Taylor-Hood Q2/Q1 and Q3/Q2, on the GPU
path through the C ABI against the FP64 oracle.

The slab blocks are (q+1) x (q+1) block matrices of the patch's spatial blocks,
factored as a block LDU (left-looking, pivoting inside the diagonal blocks) and
applied as a block forward and backward substitution; the oracle inverts each
patch's whole space-time system densely.  Tolerances are those of
tests/test_gpu_parity.py: index tables bit-exact, residual and Jacobian 1e-12,
smoother, coarse solve, Chebyshev and V-cycle 1e-10, whole solves 1e-10 with the
same FGMRES iteration counts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fem import Discretisation, Problem
from oracle.patches import PatchSmoother, patch_dofs
from oracle.solver import CoarseSolver, Hierarchy, Options, chebyshev, newton_solve
from paper_2407_13997_gb300 import inputs, wrmg
from tests.oracle_problems import oracle_problem
from tests.test_gpu_parity import Setup, cuda, rel

CASES = [inputs.fourier_small(n=4, k=1, q=2, N=2, nu=0.02), inputs.fourier_small(n=4, k=1, q=3, N=2, nu=0.02),
         inputs.fourier_small(n=8, k=1, q=2, N=3, nu=0.01), inputs.fourier_small(n=4, k=2, q=2, N=2, nu=0.02),
         inputs.fourier_small(n=4, k=2, q=3, N=2, nu=0.02)]
IDS = [w.name for w in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def setup(request):
    s = Setup(request.param)
    yield s
    s.ctx.close()


def test_patch_index_tables_bit_exact(setup):
    ctx = setup.ctx
    for l, d in enumerate(setup.discs):
        assert ctx.ndofs(l) == d.ndofs
        for patch in range((d.n + 1) ** 2):
            for slab in (0, d.N - 1):
                assert np.array_equal(ctx.patch_dofs(l, patch, slab), patch_dofs(d, patch, slab))


def test_residual_and_jacobian_match_oracle(setup):
    d = setup.discs[-1]
    F = setup.ctx.vector()
    setup.ctx.residual(cuda(setup.W[-1]), F)
    assert rel(F.cpu().numpy(), d.residual(setup.W[-1])) < 1e-12
    setup.ctx.linearise(cuda(setup.W[-1]), eig=False)
    for l, dl in enumerate(setup.discs):
        x = setup.rng.standard_normal(dl.ndofs)
        y = setup.ctx.vector(l)
        setup.ctx.apply_jacobian(l, cuda(x), y)
        assert rel(y.cpu().numpy(), dl.jacobian(setup.W[l]) @ x) < 1e-12, l


def test_smoother_and_coarse_solve_match_oracle(setup):
    ctx = setup.ctx
    ctx.linearise(cuda(setup.W[-1]), eig=False)
    for l in range(1, len(setup.discs)):
        d = setup.discs[l]
        sm = PatchSmoother(d, d.jacobian(setup.W[l]))
        r = setup.rng.standard_normal(d.ndofs)
        y = ctx.vector(l)
        ctx.patch_apply(l, cuda(r), y)
        assert rel(y.cpu().numpy(), sm.apply(r)) < 1e-10, l
    d0 = setup.discs[0]
    cs = CoarseSolver(d0, d0.jacobian(setup.W[0]))
    b = setup.rng.standard_normal(d0.ndofs)
    x = ctx.vector(0)
    ctx.coarse_solve(cuda(b), x)
    assert rel(x.cpu().numpy(), cs.solve(b)) < 1e-10


def test_eigen_estimates_chebyshev_and_vcycle_match_oracle(setup):
    w, ctx = setup.w, setup.ctx
    ctx.linearise(cuda(setup.W[-1]), eig=True)
    hier = Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options())
    hier.linearise(setup.W[-1])
    for l in range(1, len(setup.discs)):
        assert abs(ctx.get_lambda(l) - hier.levels[l].lam) < 1e-10 * hier.levels[l].lam
    L = len(setup.discs) - 1
    lev = hier.levels[L]
    b = setup.rng.standard_normal(lev.disc.ndofs) * lev.free
    x0 = setup.rng.standard_normal(lev.disc.ndofs) * lev.free
    ref = chebyshev(lambda v: lev.J @ v, lev.smoother.apply, b, x0, lev.lam, hier.opts)
    xg = cuda(x0.copy())
    ctx.smooth(L, cuda(b), xg, zero_guess=False)
    assert rel(xg.cpu().numpy(), ref) < 1e-10
    xv = ctx.vector()
    ctx.vcycle(cuda(b), xv)
    assert rel(xv.cpu().numpy(), hier.vcycle(b)) < 1e-10


@pytest.mark.parametrize("w", [inputs.fourier_small(n=4, k=1, q=2, N=3, nu=0.02),
                               inputs.poly_small(n=4, k=1, q=3, N=2), inputs.poly_small(n=4, k=2, q=2, N=2)],
                         ids=["fourier_q2q1_dg2", "poly_q2q1_dg3", "poly_q3q2_dg2"])
def test_full_solve_matches_oracle(w):
    # the polynomial solution is solved to 1e-12 so that its exactness shows
    rtol = 1e-12 if w.kind == inputs.KIND_POLY else 1e-8
    ctx = wrmg.Context(w, wrmg.default_options(newton_rtol=rtol))
    U = ctx.vector()
    ctx.initial_guess(U)
    st = ctx.solve(U)
    hier = Hierarchy(w.n_fine, w.n_coarse, w.k, w.q, w.N, oracle_problem(w), Options(newton_rtol=rtol))
    ost = {}
    ref = newton_solve(hier, stats=ost)
    assert st["gmres"] == ost["gmres"]
    assert rel(U.cpu().numpy(), ref) < 1e-10
    assert st["residuals"][-1] <= rtol * st["residuals"][0]
    ctx.close()
    if w.kind == inputs.KIND_POLY:  # u = (y^2, x^2)(1+t), p = x+y-1 lies in the discrete space
        d = Discretisation(w.n_fine, w.k, w.q, w.N, oracle_problem(w))
        ex = d.interpolant()
        free = ~d.dirichlet_mask()
        vel = np.zeros(d.ndofs, dtype=bool)
        for n in range(d.N):
            for a in range(d.nt):
                vel[d.block(n, a):d.block(n, a) + d.off_p] = True
        assert np.abs(U.cpu().numpy() - ex)[vel & free].max() < 1e-9


@pytest.mark.parametrize("q,rate", [(2, 32.0), (3, 128.0)])
def test_end_value_converges_at_order_2q_plus_1_on_the_gpu(q, rate):
    """Radau IIA superconvergence of the end value (linear Stokes, Taylor-Green decay,
    conv = 0): halving the slab width from T to T/2 divides the error at t = T by
    about 2^(2q+1).  The reference is N = 24 slabs on the same 4x4 Q2/Q1 mesh, so the
    spatial error cancels; every solve runs Newton-FGMRES-WRMG on the GPU to 1e-13."""
    def end_value(N):
        w = inputs.Workload(f"tg_linear_dg{q}_N{N}", 4, 2, 1, q, N, 0.25, 1.0 / np.pi ** 2, 0.0,
                            inputs.KIND_TAYLOR_GREEN)
        ctx = wrmg.Context(w, wrmg.default_options(newton_rtol=1e-13, ew=0, eta_fixed=1e-13))
        U = ctx.vector()
        ctx.initial_guess(U)
        ctx.solve(U)
        d = Discretisation(4, 1, q, N, oracle_problem(w))
        off = d.block(N - 1, d.nt - 1)
        out = U.cpu().numpy()[off:off + d.off_p]
        ctx.close()
        return out
    ref = end_value(24)
    e1, e2 = (np.abs(end_value(N) - ref).max() for N in (1, 2))
    assert abs((e1 / e2) / rate - 1.0) < 0.15, (e1, e2, e1 / e2)
