"""Thin ctypes binding of libwrmg (the C ABI declared in include/wrmg.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Vectors are torch CUDA float64 tensors (contiguous), passed as raw
device pointers on the current torch stream unless a stream is given.  There
is no CPU fallback: if the library is missing this module raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libwrmg.so")

WR_OK = 0
WR_ERR_ARG, WR_ERR_NOMEM, WR_ERR_CUDA, WR_ERR_NOT_CONVERGED, WR_ERR_TIMEOUT, WR_ERR_NAN, WR_ERR_STATE, \
    WR_ERR_CANCELLED = range(1, 9)
WR_FP64, WR_FP32, WR_BF16 = 0, 1, 2
WR_PATCH_SUBMATRIX, WR_PATCH_LOCAL = 0, 1
WR_WEIGHT_ONE, WR_WEIGHT_MULTIPLICITY = 0, 1
WR_RECOMPUTE, WR_STORE, WR_STORE_AUTO = 0, 1, 2
_STATUS = {1: "WR_ERR_ARG", 2: "WR_ERR_NOMEM", 3: "WR_ERR_CUDA", 4: "WR_ERR_NOT_CONVERGED",
           5: "WR_ERR_TIMEOUT", 6: "WR_ERR_NAN", 7: "WR_ERR_STATE", 8: "WR_ERR_CANCELLED"}


class WrmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("n_fine", ctypes.c_int), ("n_coarse", ctypes.c_int), ("k", ctypes.c_int), ("q", ctypes.c_int),
                ("n_slabs", ctypes.c_int), ("T", ctypes.c_double), ("nu", ctypes.c_double),
                ("conv", ctypes.c_double), ("kind", ctypes.c_int), ("steady", ctypes.c_int),
                ("n_modes", ctypes.c_int), ("mx", ctypes.POINTER(ctypes.c_int)),
                ("my", ctypes.POINTER(ctypes.c_int)), ("amp", ctypes.POINTER(ctypes.c_double)),
                ("t0", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cheb_steps", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("eig_steps", ctypes.c_int), ("newton_rtol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int), ("ew", ctypes.c_int), ("eta_fixed", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("patch_assembly", ctypes.c_int), ("scatter_weight", ctypes.c_int),
                ("store_factors", ctypes.c_int), ("recompute_slabs", ctypes.c_int),
                ("memory_budget_mb", ctypes.c_int), ("autotune", ctypes.c_int),
                ("apply_tile", ctypes.c_int), ("newton_divtol", ctypes.c_double), ("newton_stall", ctypes.c_int),
                ("time_parallel", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int * 64),
                ("residual_norms", ctypes.c_double * 65), ("setup_ms", ctypes.c_double),
                ("krylov_ms", ctypes.c_double), ("vcycles", ctypes.c_int)]

    def as_dict(self):
        n = self.newton_its
        return {"newton_its": n, "gmres": list(self.gmres_its[:n]),
                "residuals": list(self.residual_norms[:n + 1]), "setup_ms": self.setup_ms,
                "krylov_ms": self.krylov_ms, "vcycles": self.vcycles}


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "wr_default_options": (None, [ctypes.POINTER(Options)]),
    "wr_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Problem), ctypes.POINTER(Options), _P]),
    "wr_estimate_bytes": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.POINTER(Options),
                                         ctypes.POINTER(ctypes.c_int64)]),
    "wr_destroy": (ctypes.c_int, [_P]),
    "wr_last_error": (ctypes.c_char_p, [_P]),
    "wr_num_levels": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "wr_ndofs": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "wr_device_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "wr_factor_storage": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "wr_apply_tile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "wr_patch_dofs": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int)]),
    "wr_initial_guess": (ctypes.c_int, [_P, _P]),
    "wr_residual": (ctypes.c_int, [_P, _P, _P]),
    "wr_linearise": (ctypes.c_int, [_P, _P]),
    "wr_linearise_no_eig": (ctypes.c_int, [_P, _P]),
    "wr_get_lambda": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "wr_set_lambda": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "wr_apply_jacobian": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "wr_patch_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "wr_smooth": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "wr_restrict": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "wr_prolong_add": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "wr_coarse_solve": (ctypes.c_int, [_P, _P, _P]),
    "wr_vcycle": (ctypes.c_int, [_P, _P, _P]),
    "wr_vcycle_host": (ctypes.c_int, [_P, _P, _P]),
    "wr_project_pressure": (ctypes.c_int, [_P, _P]),
    "wr_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(Stats)]),
    "wr_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(Stats)]),
    "wr_set_initial_state": (ctypes.c_int, [_P, _P]),
    "wr_solve_timestepping": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(Stats)]),
    "wr_measure_fp64_tflops": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "wr_launch_count": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "wr_apply_jacobian_static": (ctypes.c_int, [ctypes.POINTER(Problem), _P, _P, _P, _P]),
    "wr_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(Problem),
                                       ctypes.POINTER(Options), _P]),
    "wr_batch_destroy": (ctypes.c_int, [_P]),
    "wr_batch_last_error": (ctypes.c_char_p, [_P]),
    "wr_batch_ndofs": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "wr_batch_device_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "wr_batch_initial_guess": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    "wr_batch_linearise": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    "wr_batch_get_lambda": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "wr_batch_vcycle": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]),
    "wr_batch_vcycle_resident": (ctypes.c_int, [_P]),
    "wr_batch_set_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "wr_batch_solve": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Stats)]),
    "wr_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(Options)]),
    "wr_server_create_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_int, ctypes.POINTER(Options)]),
    "wr_server_peak_cohort": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "wr_server_destroy": (ctypes.c_int, [_P]),
    "wr_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Problem), _P, ctypes.POINTER(ctypes.c_uint64)]),
    "wr_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, _P, ctypes.POINTER(Stats),
                                      ctypes.POINTER(ctypes.c_double)]),
    "wr_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "wr_server_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "wr_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int64]),
    "wr_selftest_bounded_wait": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "wr_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "wr_profile_jacobian": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "wr_profile_smoother": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int)]),
}


def exported_symbols():
    """Names of the C entry points this binding expects (all declared in include/wrmg.h)."""
    return sorted(_SIGS)


def load(path=LIB_PATH):
    """Loads the library (fails loudly if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libwrmg.so not found at {path}: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_options(**kw):
    o = Options()
    load().wr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def measure_fp64_tflops(stream=None):
    lib = load()
    out = ctypes.c_double()
    rc = lib.wr_measure_fp64_tflops(ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if rc != WR_OK:
        raise WrmgError(rc, "FP64 probe failed")
    return out.value


def inject_alloc_failure(nth):
    """Host-side fault injection: the nth device allocation from now on fails (0 = off)."""
    load().wr_inject_alloc_failure(int(nth))


def selftest_bounded_wait(stream=None):
    """(timed_out, waited_ms) of the smoother kernels' bounded wait on a barrier nothing completes."""
    t, ms = ctypes.c_int(), ctypes.c_double()
    rc = load().wr_selftest_bounded_wait(ctypes.c_void_p(stream or 0), ctypes.byref(t), ctypes.byref(ms))
    if rc != WR_OK:
        raise WrmgError(rc, "bounded-wait self-test failed to run")
    return bool(t.value), ms.value


def launch_count():
    out = ctypes.c_int64()
    load().wr_launch_count(ctypes.byref(out))
    return out.value


def _problem(w):
    """(Problem, arrays kept alive) for a workload description."""
    mx = np.ascontiguousarray(w.mx, dtype=np.int32)
    my = np.ascontiguousarray(w.my, dtype=np.int32)
    amp = np.ascontiguousarray(w.amp, dtype=np.float64)
    p = Problem(w.n_fine, w.n_coarse, w.k, w.q, w.N, w.T, w.nu, w.conv, w.kind, int(w.steady), len(amp),
                mx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), my.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), getattr(w, "t0", 0.0))
    return p, (mx, my, amp)


def estimate_bytes(workload, options=None):
    """Device bytes a Context for `workload` would allocate (nothing is allocated)."""
    p, keep = _problem(workload)
    o = options if options is not None else default_options()
    out = ctypes.c_int64()
    rc = load().wr_estimate_bytes(ctypes.byref(p), ctypes.byref(o), ctypes.byref(out))
    if rc != WR_OK:
        raise WrmgError(rc, "wr_estimate_bytes failed")
    return out.value


class Context:
    """One space-time solve: a level hierarchy, its factors and Krylov workspace."""

    def __init__(self, workload, options=None, stream=None):
        import torch
        lib = load()
        self._lib = lib
        self.workload = workload
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._mx = np.ascontiguousarray(workload.mx, dtype=np.int32)
        self._my = np.ascontiguousarray(workload.my, dtype=np.int32)
        self._amp = np.ascontiguousarray(workload.amp, dtype=np.float64)
        p = Problem(workload.n_fine, workload.n_coarse, workload.k, workload.q, workload.N, workload.T,
                    workload.nu, workload.conv, workload.kind, int(workload.steady), len(self._amp),
                    self._mx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    self._my.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    self._amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), getattr(workload, "t0", 0.0))
        self.options = options if options is not None else default_options()
        h = ctypes.c_void_p()
        rc = lib.wr_create(ctypes.byref(h), ctypes.byref(p), ctypes.byref(self.options), ctypes.c_void_p(stream))
        self._h = h
        if rc != WR_OK:
            msg = lib.wr_last_error(h).decode() if h.value else "wr_create failed"
            if h.value:
                lib.wr_destroy(h)
            self._h = ctypes.c_void_p()
            raise WrmgError(rc, msg)
        n = ctypes.c_int()
        lib.wr_num_levels(self._h, ctypes.byref(n))
        self.num_levels = n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.wr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != WR_OK:
            raise WrmgError(rc, self._lib.wr_last_error(self._h).decode())

    @property
    def fine(self):
        return self.num_levels - 1

    def ndofs(self, level=None):
        out = ctypes.c_int64()
        self._check(self._lib.wr_ndofs(self._h, self.fine if level is None else level, ctypes.byref(out)))
        return out.value

    def device_bytes(self):
        out = ctypes.c_int64()
        self._check(self._lib.wr_device_bytes(self._h, ctypes.byref(out)))
        return out.value

    def factor_storage(self, level):
        """(stored, window_slabs) of a smoothed level."""
        st, nw = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.wr_factor_storage(self._h, level, ctypes.byref(st), ctypes.byref(nw)))
        return bool(st.value), nw.value

    def apply_tile(self, level):
        v = ctypes.c_int()
        self._check(self._lib.wr_apply_tile(self._h, level, ctypes.byref(v)))
        return v.value

    def vector(self, level=None):
        import torch
        return torch.zeros(self.ndofs(level), dtype=torch.float64, device="cuda")

    def patch_dofs(self, level, patch, slab):
        buf = (ctypes.c_int64 * 4096)()
        ln = ctypes.c_int()
        self._check(self._lib.wr_patch_dofs(self._h, level, patch, slab, buf, ctypes.byref(ln)))
        return np.array(buf[:ln.value], dtype=np.int64)

    def initial_guess(self, U):
        self._check(self._lib.wr_initial_guess(self._h, _ptr(U)))

    def residual(self, U, F):
        self._check(self._lib.wr_residual(self._h, _ptr(U), _ptr(F)))

    def linearise(self, W, eig=True):
        fn = self._lib.wr_linearise if eig else self._lib.wr_linearise_no_eig
        self._check(fn(self._h, _ptr(W)))

    def get_lambda(self, level):
        out = ctypes.c_double()
        self._check(self._lib.wr_get_lambda(self._h, level, ctypes.byref(out)))
        return out.value

    def set_lambda(self, level, lam):
        self._check(self._lib.wr_set_lambda(self._h, level, float(lam)))

    def apply_jacobian(self, level, x, y):
        self._check(self._lib.wr_apply_jacobian(self._h, level, _ptr(x), _ptr(y)))

    def patch_apply(self, level, r, y):
        self._check(self._lib.wr_patch_apply(self._h, level, _ptr(r), _ptr(y)))

    def smooth(self, level, b, x, zero_guess):
        self._check(self._lib.wr_smooth(self._h, level, _ptr(b), _ptr(x), int(bool(zero_guess))))

    def restrict(self, fine_level, xf, xc):
        self._check(self._lib.wr_restrict(self._h, fine_level, _ptr(xf), _ptr(xc)))

    def prolong_add(self, fine_level, xc, xf):
        self._check(self._lib.wr_prolong_add(self._h, fine_level, _ptr(xc), _ptr(xf)))

    def coarse_solve(self, b, x):
        self._check(self._lib.wr_coarse_solve(self._h, _ptr(b), _ptr(x)))

    def vcycle(self, b, x):
        self._check(self._lib.wr_vcycle(self._h, _ptr(b), _ptr(x)))

    def vcycle_host(self, b, x):
        """b, x: numpy float64 arrays (pinned or pageable host memory)."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        self._check(self._lib.wr_vcycle_host(self._h, ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data)))

    def project_pressure(self, x):
        self._check(self._lib.wr_project_pressure(self._h, _ptr(x)))

    def profile(self, enable):
        self._check(self._lib.wr_profile(self._h, int(bool(enable))))

    def profile_smoother(self, level):
        ms, n = ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.wr_profile_smoother(self._h, level, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def profile_jacobian(self, level):
        """(total ms, launches, FP64 operations per launch) of the J(W) x element kernel."""
        ms, n, fl = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.wr_profile_jacobian(self._h, level, ctypes.byref(ms), ctypes.byref(n),
                                                  ctypes.byref(fl)))
        return ms.value, n.value, fl.value

    def solve(self, U, check=True):
        """Newton solve in place; the returned statistics carry the status code."""
        st = Stats()
        rc = self._lib.wr_solve(self._h, _ptr(U), ctypes.byref(st))
        if check:
            self._check(rc)
        d = st.as_dict()
        d["status"] = rc
        return d

    def set_initial_state(self, u0):
        """u0: a CUDA float64 spatial block of the finest level (length S), or None."""
        self._check(self._lib.wr_set_initial_state(self._h, _ptr(u0) if u0 is not None else None))

    def solve_timestepping(self, U, n_steps, check=True):
        """The timestepping comparator on a one-slab context; U holds n_steps slabs."""
        st = Stats()
        rc = self._lib.wr_solve_timestepping(self._h, int(n_steps), _ptr(U), ctypes.byref(st))
        if check:
            self._check(rc)
        n = min(int(n_steps), 64)
        return {"status": rc, "newton_its": st.newton_its, "vcycles": st.vcycles, "setup_ms": st.setup_ms,
                "krylov_ms": st.krylov_ms, "gmres_per_step": list(st.gmres_its[:n]),
                "final_residual_per_step": list(st.residual_norms[:n])}

    def solve_host(self, U, check=True):
        st = Stats()
        rc = self._lib.wr_solve_host(self._h, ctypes.c_void_p(U.ctypes.data), ctypes.byref(st))
        if check:
            self._check(rc)
        return st.as_dict()


class Batch:
    """Many independent solves advanced in lock step (one k and q per batch)."""

    def __init__(self, workloads, options=None, stream=None):
        import torch
        lib = load()
        self._lib = lib
        self.workloads = list(workloads)
        n = len(self.workloads)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._keep = []
        probs = (Problem * n)()
        for i, w in enumerate(self.workloads):
            mx = np.ascontiguousarray(w.mx, dtype=np.int32)
            my = np.ascontiguousarray(w.my, dtype=np.int32)
            amp = np.ascontiguousarray(w.amp, dtype=np.float64)
            self._keep += [mx, my, amp]
            probs[i] = Problem(w.n_fine, w.n_coarse, w.k, w.q, w.N, w.T, w.nu, w.conv, w.kind, int(w.steady),
                               len(amp), mx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               my.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               amp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), getattr(w, "t0", 0.0))
        self.options = options if options is not None else default_options()
        h = ctypes.c_void_p()
        rc = lib.wr_batch_create(ctypes.byref(h), n, probs, ctypes.byref(self.options), ctypes.c_void_p(stream))
        self._h = h
        if rc != WR_OK:
            msg = lib.wr_batch_last_error(h).decode() if h.value else "wr_batch_create failed"
            if h.value:
                lib.wr_batch_destroy(h)
            self._h = ctypes.c_void_p()
            raise WrmgError(rc, msg)
        self.n = n

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.wr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != WR_OK:
            raise WrmgError(rc, self._lib.wr_batch_last_error(self._h).decode())

    @staticmethod
    def _ptrs(ts):
        for t in ts:
            _ptr(t)
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def ndofs(self, m):
        out = ctypes.c_int64()
        self._check(self._lib.wr_batch_ndofs(self._h, m, ctypes.byref(out)))
        return out.value

    def device_bytes(self):
        out = ctypes.c_int64()
        self._check(self._lib.wr_batch_device_bytes(self._h, ctypes.byref(out)))
        return out.value

    def vectors(self):
        import torch
        return [torch.zeros(self.ndofs(m), dtype=torch.float64, device="cuda") for m in range(self.n)]

    def initial_guess(self, Us):
        self._check(self._lib.wr_batch_initial_guess(self._h, self._ptrs(Us)))

    def linearise(self, Ws):
        self._check(self._lib.wr_batch_linearise(self._h, self._ptrs(Ws)))

    def get_lambda(self, m, level):
        out = ctypes.c_double()
        self._check(self._lib.wr_batch_get_lambda(self._h, m, level, ctypes.byref(out)))
        return out.value

    def vcycle(self, bs, xs):
        self._check(self._lib.wr_batch_vcycle(self._h, self._ptrs(bs), self._ptrs(xs)))

    def set_graphs(self, enable):
        self._check(self._lib.wr_batch_set_graphs(self._h, int(bool(enable))))

    def vcycle_resident(self):
        self._check(self._lib.wr_batch_vcycle_resident(self._h))

    def solve(self, Us, check=True):
        st = (Stats * self.n)()
        rc = self._lib.wr_batch_solve(self._h, self._ptrs(Us), st)
        if check:
            self._check(rc)
        return [s.as_dict() for s in st]


class Server:
    """A request loop over independent solves: FIFO admission under a device
    memory budget and an in-flight cap.  batch_members = 1: each admitted request
    runs on its own native worker thread, CUDA stream and context; > 1: each
    in-flight slot solves a cohort of up to batch_members queued requests (same k
    and q) as one lock-step batch (wr_server_create_batched)."""

    def __init__(self, mem_budget_bytes, max_inflight, options=None, batch_members=1):
        lib = load()
        self._lib = lib
        self.options = options if options is not None else default_options()
        h = ctypes.c_void_p()
        if batch_members > 1:
            rc = lib.wr_server_create_batched(ctypes.byref(h), int(mem_budget_bytes), int(max_inflight),
                                              int(batch_members), ctypes.byref(self.options))
        else:
            rc = lib.wr_server_create(ctypes.byref(h), int(mem_budget_bytes), int(max_inflight),
                                      ctypes.byref(self.options))
        if rc != WR_OK:
            raise WrmgError(rc, "wr_server_create failed")
        self._h = h
        self._ndofs = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.wr_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, workload, U0=None):
        """Queues one solve; returns its ticket.  U0: optional host float64 iterate."""
        p, keep = _problem(workload)
        ptr = None
        if U0 is not None:
            U0 = np.ascontiguousarray(U0, dtype=np.float64)
            ptr = ctypes.c_void_p(U0.ctypes.data)
        t = ctypes.c_uint64()
        rc = self._lib.wr_server_submit(self._h, ctypes.byref(p), ptr, ctypes.byref(t))
        if rc != WR_OK:
            raise WrmgError(rc, "wr_server_submit failed")
        self._ndofs[t.value] = workload.ndofs()
        return t.value

    def poll(self, ticket, wait=True, want_solution=True):
        """None while the request runs (wait=False); else (status, U or None, stats, latency_ms)."""
        n = self._ndofs[ticket]
        U = np.empty(n, dtype=np.float64) if want_solution else None
        st = Stats()
        lat = ctypes.c_double()
        rc = self._lib.wr_server_poll(self._h, ctypes.c_uint64(ticket), int(bool(wait)),
                                      ctypes.c_void_p(U.ctypes.data) if U is not None else None,
                                      ctypes.byref(st), ctypes.byref(lat))
        if rc == WR_ERR_STATE and not wait:
            return None
        del self._ndofs[ticket]
        return rc, U, st.as_dict(), lat.value

    def cancel(self, ticket):
        rc = self._lib.wr_server_cancel(self._h, ctypes.c_uint64(ticket))
        if rc != WR_OK:
            raise WrmgError(rc, "wr_server_cancel failed")

    def stats(self):
        b, n, c = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        self._lib.wr_server_stats(self._h, ctypes.byref(b), ctypes.byref(n))
        self._lib.wr_server_peak_cohort(self._h, ctypes.byref(c))
        return {"peak_bytes": b.value, "peak_inflight": n.value, "peak_cohort": c.value}
