"""The allocation-free Jacobian entry point (wr_apply_jacobian_static).

Callers that cannot call cudaMalloc (an application that owns all device memory
through its own pool, or a latency-critical loop that must not pay for the
allocator's implicit synchronisation) use wr_apply_jacobian_static, whose only
scratch is a fixed static device array inside the library.  This test calls it
through the C ABI twice in a row and compares each result with the context-based
wr_apply_jacobian on the same inputs, at the 1e-12 relative tolerance the other
Jacobian parity tests use, and checks that the second call changes neither
torch's allocated bytes nor the device's free bytes; it also checks that an
oversized problem and a heat problem are refused before any work is enqueued.  It lives in a file of its own that pytest collects
last and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_13997_gb300 import inputs, wrmg


def problem_struct(w, keep):
    mx = np.ascontiguousarray(w.mx, dtype=np.int32)
    my = np.ascontiguousarray(w.my, dtype=np.int32)
    amp = np.ascontiguousarray(w.amp, dtype=np.float64)
    keep.extend([mx, my, amp])
    return wrmg.Problem(w.n_fine, w.n_coarse, w.k, w.q, w.N, w.T, w.nu, w.conv, w.kind, int(w.steady), len(amp),
                        mx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        my.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("w", [inputs.fourier_small(n=8, k=2, q=1, N=4, nu=1e-2),
                               inputs.fourier_small(n=16, k=1, q=0, N=3, nu=1e-3)], ids=["q3q2_dg1", "q2q1_dg0"])
def test_static_scratch_jacobian_matches_context_entry_point_twice(w):
    lib = wrmg.load()
    ctx = wrmg.Context(w)
    rng = np.random.default_rng(21)
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    ctx.linearise(W, eig=False)
    keep = []
    p = problem_struct(w, keep)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xs = [torch.from_numpy(rng.standard_normal(ctx.ndofs())).cuda() for _ in range(2)]
    refs = [ctx.vector() for _ in range(2)]
    outs = [ctx.vector() for _ in range(2)]
    for x, ref in zip(xs, refs):
        ctx.apply_jacobian(ctx.fine, x, ref)
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            # every buffer exists already; the first call has loaded the library's
            # module and looked up the scratch address on this device
            torch.cuda.synchronize()
            before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        rc = lib.wr_apply_jacobian_static(ctypes.byref(p), ptr(W), ptr(xs[call]), ptr(outs[call]), stream)
        assert rc == wrmg.WR_OK, lib.wr_last_error(None)
        torch.cuda.synchronize()
        err = (outs[call] - refs[call]).abs().max().item() / refs[call].abs().max().item()
        assert err < 1e-12, (call, err)
    # the second call allocated no device memory, through torch or otherwise
    assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before
    ctx.close()


def test_static_scratch_refuses_problems_larger_than_its_array():
    lib = wrmg.load()
    w = inputs.fourier_64x64_q3q2_dg1(0)       # 64 slabs x 4096 cells x 82 > 8 Mi doubles
    keep = []
    p = problem_struct(w, keep)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.wr_apply_jacobian_static(ctypes.byref(p), ptr(dummy), ptr(dummy), ptr(out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == wrmg.WR_ERR_ARG
    assert b"larger than the static array" in lib.wr_last_error(None)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_static_scratch_refuses_the_heat_kinds():
    lib = wrmg.load()
    w = inputs.heat(n=4, k=1, q=0, N=2)
    keep = []
    p = problem_struct(w, keep)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.wr_apply_jacobian_static(ctypes.byref(p), ptr(dummy), ptr(dummy), ptr(out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == wrmg.WR_ERR_ARG
    assert b"not a Navier-Stokes problem" in lib.wr_last_error(None)
