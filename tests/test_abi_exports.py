"""The C-ABI library loads and exports every entry point include/wrmg.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wrmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(wr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_13997_gb300 import build, wrmg
    if not os.path.exists(wrmg.LIB_PATH):
        build.build()
    return wrmg.LIB_PATH


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ["wr_create", "wr_destroy", "wr_residual", "wr_linearise", "wr_apply_jacobian", "wr_patch_apply",
                 "wr_smooth", "wr_restrict", "wr_prolong_add", "wr_vcycle", "wr_solve", "wr_patch_dofs",
                 "wr_ndofs", "wr_num_levels", "wr_initial_guess", "wr_coarse_solve"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header_and_loads(libpath):
    from paper_2407_13997_gb300 import wrmg
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert set(wrmg.exported_symbols()) == set(declared_functions())
    o = wrmg.default_options()
    assert o.cheb_steps == 2 and o.eig_steps == 10 and abs(o.cheb_lo - 0.25) < 1e-15 and o.gmres_restart == 30


def test_allocation_estimate_runs_on_the_host(libpath):
    # the dry run of wr_create makes no CUDA call, so it works without a GPU
    from paper_2407_13997_gb300 import inputs, wrmg
    w = inputs.fourier_64x64_q3q2_dg1()
    e = {p: wrmg.estimate_bytes(w, wrmg.default_options(precision=p)) for p in (wrmg.WR_FP64, wrmg.WR_FP32,
                                                                                 wrmg.WR_BF16)}
    # the fine-level factors alone: one (q+1) MS x (q+1) MS block per patch and slab, MS = 107 for k = 2
    npatch, ms, nt = 65 * 65, 107, 2
    fine_factors = npatch * w.N * (nt * ms) ** 2
    assert e[wrmg.WR_FP64] > 8 * fine_factors
    assert e[wrmg.WR_FP64] > e[wrmg.WR_FP32] > e[wrmg.WR_BF16] > 2 * fine_factors
    assert e[wrmg.WR_FP64] - e[wrmg.WR_FP32] > 4 * fine_factors
    # doubling the slab count roughly doubles everything that scales with N
    w2 = inputs.fourier_64x64_q3q2_dg1()
    w2.N = 128
    assert 1.9 < wrmg.estimate_bytes(w2) / e[wrmg.WR_FP64] < 2.05
    bad = inputs.fourier_small(n=8, k=1, q=0, N=3, nu=0.02)
    bad.k = 3
    with pytest.raises(wrmg.WrmgError):
        wrmg.estimate_bytes(bad)


def test_store_or_recompute_plan_on_the_host(libpath):
    """The planner of wr_create (run dry by wr_estimate_bytes): recomputing the
    factors needs far less memory than storing them, and the automatic choice keeps
    the fewest recomputing levels that fit the budget."""
    from paper_2407_13997_gb300 import inputs, wrmg
    w = inputs.fourier_64x64_q3q2_dg1()
    est = lambda **kw: wrmg.estimate_bytes(w, wrmg.default_options(**kw))
    store = est(store_factors=wrmg.WR_STORE)
    rec = est(store_factors=wrmg.WR_RECOMPUTE, recompute_slabs=4)
    assert rec < store / 4
    mib = lambda b: int(b // (1 << 20)) + 1
    assert est(store_factors=wrmg.WR_STORE_AUTO) == store                     # no budget given: store
    assert est(store_factors=wrmg.WR_STORE_AUTO, memory_budget_mb=mib(store)) == store
    mid = (store + rec) // 2
    auto = est(store_factors=wrmg.WR_STORE_AUTO, memory_budget_mb=mib(mid), recompute_slabs=4)
    assert rec <= auto <= mid + (1 << 20)
    assert est(store_factors=wrmg.WR_STORE_AUTO, memory_budget_mb=1, recompute_slabs=4) == rec


def test_heat_degrees_and_coarse_mesh_checks_on_the_host(libpath):
    """The heat equation takes Q_k x DG(q) for k = 1..3, q = 0..3 (Sec. 5); its stored
    factors are one (q+1)(2k-1)^2 block per patch and slab, FP64.  The k = q = 3 coarse
    block of a 2x2 mesh (196 x 196) does not fit the direct solve and is refused; the 1x1
    coarse mesh is taken instead.  Navier-Stokes takes DG(2) and DG(3) with FP64 factors
    only."""
    from paper_2407_13997_gb300 import inputs, wrmg
    for k in (1, 2, 3):
        for q in (0, 1, 2, 3):
            w = inputs.heat(n=16, k=k, q=q, N=4)
            m = (q + 1) * (2 * k - 1) ** 2
            fine_factors = 17 * 17 * 4 * m * m * 8
            assert wrmg.estimate_bytes(w) > fine_factors
    assert inputs.heat(k=3, q=3).n_coarse == 1
    bad = inputs.heat(n=16, k=3, q=3, N=4, n_coarse=2)
    with pytest.raises(wrmg.WrmgError):
        wrmg.estimate_bytes(bad)
    ns = inputs.fourier_small(n=8, k=1, q=0, N=3)
    for q in (2, 3):
        ns.q = q
        assert wrmg.estimate_bytes(ns) > 0
        with pytest.raises(wrmg.WrmgError):
            wrmg.estimate_bytes(ns, wrmg.default_options(precision=wrmg.WR_FP32))
    ns3 = inputs.fourier_small(n=8, k=2, q=0, N=3)
    ns3.q = 2
    assert wrmg.estimate_bytes(ns3) > 0
    with pytest.raises(wrmg.WrmgError):
        wrmg.estimate_bytes(ns3, wrmg.default_options(precision=wrmg.WR_BF16))
    ns3.q = 4
    with pytest.raises(wrmg.WrmgError):
        wrmg.estimate_bytes(ns3)
