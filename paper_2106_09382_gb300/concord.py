"""Python binding of the C ABI in ``include/concord.h`` (ctypes).

Argument marshalling only: every step of the estimator runs in the CUDA
library ``libconcord_gb300.so``.  Device buffers are torch tensors (used for
memory and streams only); host buffers are numpy arrays.  Loading raises if
the library cannot be built or loaded: there is no CPU fallback.

Names follow the C entry points: ``concord_schedule``, ``concord_gram``,
``State`` (concord_create / _set_S / _set_omega / _sweep / _run /
_solve_device / _solve_host / _get_omega / _get_W / _get_history /
_lambda_max / _set_timeout / _set_fault / _destroy), ``concord_solve`` and
``Joint`` (the concord_joint_* entry points of the two-population joint
estimator).
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

OK, NOT_CONVERGED = 0, 1
E_ARG, E_NONPOS_DIAG, E_NONFINITE, E_CUDA, E_TIMEOUT, E_NOMEM, E_OCCUPANCY = (
    -1, -2, -3, -4, -5, -6, -7)
FP64, MIXED = 0, 1
F64, F32 = 0, 1
PREP_NONE, PREP_CENTER, PREP_STANDARDIZE = 0, 1, 2
GRAM_FP64, GRAM_FP32, GRAM_TF32X3, GRAM_BF16X3 = 0, 1, 2, 3
STOP_KKT, STOP_DELTA = 0, 1
SWEEP_AUTO, SWEEP_GRID, SWEEP_CLUSTER, SWEEP_SCREENED, SWEEP_DENSE = 0, 1, 2, 3, 4
JOINT_ROWFLAGS, JOINT_BARRIER = 0, 1

STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "E_ARG", -2: "E_NONPOS_DIAG",
                -3: "E_NONFINITE", -4: "E_CUDA", -5: "E_TIMEOUT", -6: "E_NOMEM",
                -7: "E_OCCUPANCY"}


class ConcordResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("sweeps_fp32", ctypes.c_int), ("first_delta_sweep", ctypes.c_int),
                ("objective", ctypes.c_double), ("kkt", ctypes.c_double),
                ("delta", ctypes.c_double), ("lam", ctypes.c_double),
                ("active_pairs", ctypes.c_longlong), ("seconds", ctypes.c_double),
                ("timeout_vertex", ctypes.c_int), ("timeout_step", ctypes.c_int),
                ("screen_redos", ctypes.c_int), ("dense_sweeps", ctypes.c_int),
                ("s_refined", ctypes.c_int), ("lazy_sweeps", ctypes.c_int),
                ("sparse_sweeps", ctypes.c_int), ("partial_sweeps", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class AdjointInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("active_pairs", ctypes.c_longlong), ("residual", ctypes.c_double),
                ("dlambda", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ConcordError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


_vp, _ci, _cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_rp = ctypes.POINTER(ConcordResult)
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (argtypes, restype); the exported symbols of include/concord.h
SIGNATURES = {
    "concord_result_size": ([], ctypes.c_size_t),
    "concord_last_error": ([], ctypes.c_char_p),
    "concord_version": ([], ctypes.c_char_p),
    "concord_schedule": ([_ci, ctypes.POINTER(ctypes.c_int32), _ip], _ci),
    "concord_gram": ([_vp, _ci, _ci, _ci, _ci, _ci, _ci, _vp, _ci, _ci, _vp], _ci),
    "concord_gram_static": ([_vp, _ci, _ci, _ci, _ci, _ci, _vp, _ci, _vp], _ci),
    "concord_create": ([ctypes.POINTER(_vp), _ci, _ci, _ci, _ci], _ci),
    "concord_destroy": ([_vp], _ci),
    "concord_set_stream": ([_vp, _vp], _ci),
    "concord_set_timeout": ([_vp, _cd], _ci),
    "concord_set_S": ([_vp, _vp, _ci, _ci], _ci),
    "concord_set_omega": ([_vp, _vp, _ci, _ci], _ci),
    "concord_get_omega": ([_vp, _vp, _ci, _ci], _ci),
    "concord_get_W": ([_vp, _vp, _ci, _ci], _ci),
    "concord_get_history": ([_vp, _dp, _ci, _ip], _ci),
    "concord_set_gram_mode": ([_vp, _ci], _ci),
    "concord_set_refine": ([_vp, _ci], _ci),
    "concord_set_lazy_verify": ([_vp, _ci], _ci),
    "concord_set_sparse_polish": ([_vp, _ci], _ci),
    "concord_autotune": ([_vp, _cd, _cd, _ci, _dp, _ip, _ip], _ci),
    "concord_set_rows_per_warp": ([_vp, _ci], _ci),
    "concord_set_sweep_variant": ([_vp, _ci], _ci),
    "concord_set_poll_sleep": ([_vp, _ci], _ci),
    "concord_get_sweep_variant": ([_vp, _ip, _ip], _ci),
    "concord_sweep": ([_vp, _cd, _ci, _rp], _ci),
    "concord_run": ([_vp, _cd, _cd, _ci, _ci, _cd, _rp], _ci),
    "concord_solve_device": ([_vp, _vp, _ci, _ci, _ci, _ci, _cd, _cd, _ci, _ci, _vp, _ci, _ci,
                              _rp], _ci),
    "concord_solve_host": ([_vp, _dp, _ci, _ci, _cd, _cd, _ci, _ci, _dp, _rp], _ci),
    "concord_solve": ([_dp, _ci, _ci, _ci, _ci, _cd, _cd, _ci, _ci, _dp, _dp, _rp], _ci),
    "concord_lambda_max": ([_vp, _dp], _ci),
    "concord_set_fault": ([_vp, _ci, _ci], _ci),
    "concord_get_timing": ([_vp, _dp, _ip, _ci, _ip], _ci),
    "concord_kernel_launches": ([], ctypes.c_ulonglong),
    "concord_path": ([_vp, _dp, _ci, _cd, _ci, _rp, _vp, _ci], _ci),
    "concord_stability": ([_vp, _vp, _ci, _ci, _ci, _ci, _ip, _ip, _ci, _dp, _ci, _cd, _ci, _ci,
                           _vp], _ci),
    "concord_get_omega_csr": ([_vp, _ip, _ip, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
                              _ci),
    "concord_heldout": ([_vp, _vp, _ci, _ci, _dp], _ci),
    "concord_adjoint": ([_vp, _vp, _ci, _ci, _cd, _ci, _vp, _ci, ctypes.POINTER(AdjointInfo)], _ci),
    "concord_adjoint_data": ([_vp, _vp, _ci, _ci, _ci, _ci, _vp, _ci, _ci], _ci),
    "concord_tune_lambda": ([_vp, _vp, _ci, _ci, _cd, _ci, _cd, _cd, _ci, _cd, _dp], _ci),
    "concord_joint_create": ([ctypes.POINTER(_vp), _ci, _ci, _ci], _ci),
    "concord_joint_destroy": ([_vp], _ci),
    "concord_joint_set_stream": ([_vp, _vp], _ci),
    "concord_joint_set_timeout": ([_vp, _cd], _ci),
    "concord_joint_set_grid": ([_vp, _ci], _ci),
    "concord_joint_set_variant": ([_vp, _ci], _ci),
    "concord_joint_set_fault": ([_vp, _ci, _ci], _ci),
    "concord_joint_set_S": ([_vp, _ci, _vp, _ci, _ci], _ci),
    "concord_joint_set_omega": ([_vp, _ci, _vp, _ci, _ci], _ci),
    "concord_joint_get_omega": ([_vp, _ci, _vp, _ci, _ci], _ci),
    "concord_joint_sweep": ([_vp, _cd, _cd, _ci, _rp], _ci),
    "concord_joint_run": ([_vp, _cd, _cd, _cd, _ci, _rp], _ci),
    "concord_joint_get_history": ([_vp, _dp, _ci, _ip], _ci),
}

SIGNATURES.update({
    "concord_batch_create": ([ctypes.POINTER(_vp), _ci, _ip, _ci, _ci, _ci], _ci),
    "concord_batch_destroy": ([_vp], _ci),
    "concord_batch_set_stream": ([_vp, _vp], _ci),
    "concord_batch_set_timeout": ([_vp, _cd], _ci),
    "concord_batch_set_S": ([_vp, _ci, _vp, _ci, _ci], _ci),
    "concord_batch_gram": ([_vp, _ci, _vp, _ci, _ci, _ci, _vp, _ci, _ci], _ci),
    "concord_batch_reset": ([_vp, _ci], _ci),
    "concord_batch_path": ([_vp, _dp, _ci, _cd, _ci, _rp, _vp], _ci),
    "concord_batch_set_rows_per_warp": ([_vp, _ci], _ci),
    "concord_batch_set_polish": ([_vp, _ci], _ci),
    "concord_batch_autotune": ([_vp, _cd, _ci, _dp], _ci),
    "concord_batch_info": ([_vp, _ip, _ip, _ip, _dp], _ci),
    "concord_batch_get_omega": ([_vp, _ci, _vp, _ci, _ci], _ci),
})

_lock = threading.Lock()
_lib = None


def load(build: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) libconcord_gb300.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if lib.concord_result_size() != ctypes.sizeof(ConcordResult):
            raise RuntimeError("concord_result layout mismatch")
        _lib = lib
        return lib


def _check(rc: int, allow=(OK,)) -> int:
    if rc in allow:
        return rc
    msg = load().concord_last_error().decode(errors="replace")
    raise ConcordError(rc, msg)


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().concord_kernel_launches())


def last_error() -> str:
    return load().concord_last_error().decode(errors="replace")


# ------------------------------------------------------------------ schedule
def concord_schedule(p: int) -> np.ndarray:
    """(pe-1, pe/2, 2) int32 pairs of the circle-method colouring (Section 3.2)."""
    pe = p + (p % 2)
    out = np.empty((max(pe - 1, 1), max(pe // 2, 1), 2), dtype=np.int32)
    nc = ctypes.c_int(0)
    _check(load().concord_schedule(int(p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ctypes.byref(nc)))
    return out


# ---------------------------------------------------------------------- gram
def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("float64 or float32 tensor expected, got %s" % t.dtype)


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def concord_gram(X, prep: int = PREP_STANDARDIZE, mode: int = GRAM_FP64, out_dtype=None,
                 stream=None):
    """S = Z^T Z / n on the device for a CUDA tensor X (n x p, row-major)."""
    import torch
    assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
    n, p = X.shape
    out_dtype = out_dtype or (torch.float64 if mode == GRAM_FP64 else torch.float32)
    with torch.cuda.device(X.device):
        S = torch.empty((p, p), dtype=out_dtype, device=X.device)
        _check(load().concord_gram(X.data_ptr(), _dtype_code(X), n, p, X.stride(0), prep, mode,
                                   S.data_ptr(), _dtype_code(S), p, _stream_ptr(stream)))
    return S


def concord_gram_static(X, prep: int = PREP_STANDARDIZE, out=None, stream=None):
    """FP64 S = Z^T Z / n through the allocation-free entry point (the device
    statistics live in the library's fixed array; p <= 16384).  `out` may
    give the p x p float64 output tensor on X's device (row stride >= p).
    The call runs with X's device current, on `stream` or that device's
    current stream."""
    import torch
    assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
    n, p = X.shape
    with torch.cuda.device(X.device):
        if out is None:
            S = torch.empty((p, p), dtype=torch.float64, device=X.device)
        else:
            S = out
            if S.device != X.device:
                raise ValueError("out is on %s, X on %s" % (S.device, X.device))
            if S.dtype != torch.float64 or S.dim() != 2 or tuple(S.shape) != (p, p):
                raise ValueError("out must be a (%d, %d) float64 tensor" % (p, p))
            if S.stride(1) != 1 or S.stride(0) < p:
                raise ValueError("out must have unit column stride and row stride >= p")
        _check(load().concord_gram_static(X.data_ptr(), _dtype_code(X), n, p, X.stride(0), prep,
                                          S.data_ptr(), S.stride(0), _stream_ptr(stream)))
    return S


# --------------------------------------------------------------------- state
class State:
    """A solver state (concord_create) bound to one device and stream."""

    def __init__(self, p: int, precision: int = FP64, n_cap: int = 0, device: int | None = None):
        import torch
        lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        self._ptr = ctypes.c_void_p()
        _check(lib.concord_create(ctypes.byref(self._ptr), int(p), int(precision), int(n_cap),
                                  dev))
        self.p, self.precision, self.n_cap, self.device = int(p), int(precision), int(n_cap), dev
        self.last = None

    # lifecycle
    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            load().concord_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # configuration
    def set_stream(self, stream=None):
        _check(load().concord_set_stream(self._ptr, _stream_ptr(stream) if stream is not False
                                         else None))

    def set_timeout(self, seconds: float):
        _check(load().concord_set_timeout(self._ptr, float(seconds)))

    def set_fault(self, vertex: int, step: int = 0):
        _check(load().concord_set_fault(self._ptr, int(vertex), int(step)))

    def set_rows_per_warp(self, rows: int):
        _check(load().concord_set_rows_per_warp(self._ptr, int(rows)))

    def set_poll_sleep(self, ns: int):
        _check(load().concord_set_poll_sleep(self._ptr, int(ns)))

    def set_sweep_variant(self, variant: int):
        _check(load().concord_set_sweep_variant(self._ptr, int(variant)))

    def sweep_variant(self):
        """(variant of the last launch, largest cluster size found)."""
        v, cs = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().concord_get_sweep_variant(self._ptr, ctypes.byref(v), ctypes.byref(cs)))
        return v.value, cs.value

    def set_gram_mode(self, mode: int):
        _check(load().concord_set_gram_mode(self._ptr, int(mode)))

    # data
    AUTOTUNE_CHOICES = ("screened/0", "cluster/32", "cluster/16", "cluster/8", "cluster/4",
                        "grid/32", "grid/16", "grid/8", "grid/4")

    def autotune(self, lam: float, tol: float = 1e-5, max_sweeps: int = 1000):
        """Pick the sweep kernel / layout by measured time per sweep
        (concord_autotune); returns (choice name, {choice: ms per sweep})."""
        ms = np.zeros(len(self.AUTOTUNE_CHOICES), dtype=np.float64)
        v, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().concord_autotune(self._ptr, float(lam), float(tol), int(max_sweeps),
                                       ms.ctypes.data_as(_dp), ctypes.byref(v), ctypes.byref(r)))
        names = {SWEEP_SCREENED: "screened", SWEEP_CLUSTER: "cluster", SWEEP_GRID: "grid"}
        trial = {k: float(x) for k, x in zip(self.AUTOTUNE_CHOICES, ms) if x >= 0}
        return "%s/%d" % (names[v.value], r.value), trial

    def set_lazy_verify(self, on: bool):
        """Skip the screened kernel's verification pass when the changes
        provably keep every other pair at zero (concord_set_lazy_verify)."""
        _check(load().concord_set_lazy_verify(self._ptr, 1 if on else 0))

    def set_sparse_polish(self, on: bool):
        """Mixed states: FP64 polish on the FP32 phase's candidates without
        rebuilding W while the lazy bound holds (concord_set_sparse_polish)."""
        _check(load().concord_set_sparse_polish(self._ptr, 1 if on else 0))

    def set_refine(self, on: bool):
        """Recompute the neighbourhood's S entries in FP64 accuracy before a
        mixed solve's polish (concord_set_refine; on by default)."""
        _check(load().concord_set_refine(self._ptr, 1 if on else 0))

    def set_S(self, S):
        assert S.is_cuda and S.dim() == 2 and S.stride(1) == 1
        _check(load().concord_set_S(self._ptr, S.data_ptr(), _dtype_code(S), S.stride(0)))

    def set_omega(self, Om):
        assert Om.is_cuda and Om.dim() == 2 and Om.stride(1) == 1
        _check(load().concord_set_omega(self._ptr, Om.data_ptr(), _dtype_code(Om), Om.stride(0)))

    def get_omega(self, dtype=None):
        import torch
        out = torch.empty((self.p, self.p), dtype=dtype or torch.float64,
                          device="cuda:%d" % self.device)
        _check(load().concord_get_omega(self._ptr, out.data_ptr(), _dtype_code(out), self.p))
        return out

    def get_omega_csr(self, cap: int | None = None, out=None):
        """Omega as host CSR arrays (rowptr int32 [p+1], col int32, val
        float64).  `out` may pass preallocated (pinned) numpy arrays
        (rowptr, col, val) whose length sets the capacity."""
        lib = load()
        nnz = ctypes.c_int64(0)
        if out is not None:
            rowptr, col, val = out
            cap = len(col)
        else:
            rowptr = np.empty(self.p + 1, dtype=np.int32)
            if cap is None:
                rc = lib.concord_get_omega_csr(self._ptr, rowptr.ctypes.data_as(_ip), None, None, 0,
                                               ctypes.byref(nnz))
                _check(rc, (OK, E_ARG))
                cap = int(nnz.value)
            col = np.empty(cap, dtype=np.int32)
            val = np.empty(cap, dtype=np.float64)
        _check(lib.concord_get_omega_csr(self._ptr, rowptr.ctypes.data_as(_ip),
                                         col.ctypes.data_as(_ip), val.ctypes.data_as(_dp), int(cap),
                                         ctypes.byref(nnz)))
        k = int(nnz.value)
        return rowptr, col[:k], val[:k]

    def get_W(self, dtype=None):
        import torch
        out = torch.empty((self.p, self.p), dtype=dtype or torch.float64,
                          device="cuda:%d" % self.device)
        _check(load().concord_get_W(self._ptr, out.data_ptr(), _dtype_code(out), self.p))
        return out

    def history(self) -> np.ndarray:
        rows = ctypes.c_int(0)
        _check(load().concord_get_history(self._ptr, None, 0, ctypes.byref(rows)))
        h = np.zeros((max(rows.value, 1), 4), dtype=np.float64)
        _check(load().concord_get_history(self._ptr, h.ctypes.data_as(_dp), rows.value,
                                          ctypes.byref(rows)))
        return h[: rows.value]

    def timing(self):
        """[(milliseconds, sweeps)] of each sweep-kernel launch of the last call."""
        ms = (ctypes.c_double * 4)()
        sw = (ctypes.c_int * 4)()
        n = ctypes.c_int(0)
        _check(load().concord_get_timing(self._ptr, ms, sw, 4, ctypes.byref(n)))
        return [(ms[q], sw[q]) for q in range(min(n.value, 4))]

    def lambda_max(self) -> float:
        v = ctypes.c_double(0)
        _check(load().concord_lambda_max(self._ptr, ctypes.byref(v)))
        return v.value

    # iteration
    def sweep(self, lam: float, n_sweeps: int = 1) -> ConcordResult:
        r = ConcordResult()
        rc = load().concord_sweep(self._ptr, float(lam), int(n_sweeps), ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r

    def run(self, lam: float, tol: float = 1e-5, max_sweeps: int = 1000,
            stop_rule: int = STOP_KKT, switch_tol: float = 0.0) -> ConcordResult:
        r = ConcordResult()
        rc = load().concord_run(self._ptr, float(lam), float(tol), int(max_sweeps),
                                int(stop_rule), float(switch_tol), ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r

    def solve_device(self, X, lam: float, tol: float = 1e-5, max_sweeps: int = 1000,
                     prep: int = PREP_STANDARDIZE, stop_rule: int = STOP_KKT, Omega_out=None):
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        r = ConcordResult()
        optr, odt, old = (None, F64, self.p)
        if Omega_out is not None:
            optr, odt, old = Omega_out.data_ptr(), _dtype_code(Omega_out), Omega_out.stride(0)
        rc = load().concord_solve_device(self._ptr, X.data_ptr(), _dtype_code(X), X.shape[0],
                                         X.stride(0), int(prep), float(lam), float(tol),
                                         int(max_sweeps), int(stop_rule), optr, odt, old,
                                         ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r

    def path(self, lambdas, tol: float = 1e-5, max_sweeps: int = 1000, omega_out=None):
        """Warm-started lambda path from the current iterate; returns one
        ConcordResult per lambda.  omega_out (device tensor, n_lambda x p x
        ldo, float32 for MIXED / float64 for FP64) receives each Omega."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        res = (ConcordResult * len(lam))()
        optr, ldo = None, self.p
        if omega_out is not None:
            assert omega_out.is_cuda and omega_out.dim() == 3 and omega_out.stride(2) == 1
            optr, ldo = omega_out.data_ptr(), omega_out.stride(1)
        rc = load().concord_path(self._ptr, lam.ctypes.data_as(_dp), len(lam), float(tol),
                                 int(max_sweeps), res, optr, ldo)
        _check(rc)
        return list(res)

    def stability(self, X, subsets, lambdas, tol: float = 1e-5, max_sweeps: int = 1000,
                  prep: int = PREP_STANDARDIZE, workers: int = 0, freq_out=None):
        """Stability selection: for each row subset of X (device tensor), the
        Gram of its rows and the lambda path from Omega = I; returns the
        per-lambda edge frequencies (device float32 tensor n_lambda x p x p)."""
        import torch
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        rows = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32)
                                                    for s in subsets]), dtype=np.int32)
        sizes = np.ascontiguousarray([len(s) for s in subsets], dtype=np.int32)
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        if freq_out is None:
            freq_out = torch.empty((len(lam), self.p, self.p), dtype=torch.float32,
                                   device=X.device)
        rc = load().concord_stability(self._ptr, X.data_ptr(), _dtype_code(X), X.shape[0],
                                      X.stride(0), int(prep), rows.ctypes.data_as(_ip),
                                      sizes.ctypes.data_as(_ip), len(sizes),
                                      lam.ctypes.data_as(_dp), len(lam), float(tol),
                                      int(max_sweeps), int(workers), freq_out.data_ptr())
        _check(rc)
        return freq_out

    # implicit differentiation
    def heldout(self, S_val) -> float:
        """Held-out loss of the current Omega for the validation Gram S_val;
        its gradient on the active set becomes the next adjoint's right-hand
        side."""
        assert S_val.is_cuda and S_val.dim() == 2 and S_val.stride(1) == 1
        v = ctypes.c_double(0)
        _check(load().concord_heldout(self._ptr, S_val.data_ptr(), _dtype_code(S_val),
                                      S_val.stride(0), ctypes.byref(v)))
        return v.value

    def adjoint(self, g=None, tol: float = 1e-10, max_iter: int = 10000, dS_out=None):
        """Adjoint solve on the active set for the loss gradient g (p x p
        device tensor, full-matrix convention; None: the held-out gradient).
        Returns AdjointInfo (dL/dlambda in .dlambda); dS_out (p x p float64
        device tensor) receives dL/dS."""
        info = AdjointInfo()
        gptr, gdt, ldg = None, F64, self.p
        if g is not None:
            assert g.is_cuda and g.dim() == 2 and g.stride(1) == 1
            gptr, gdt, ldg = g.data_ptr(), _dtype_code(g), g.stride(0)
        sptr, lds = None, self.p
        if dS_out is not None:
            import torch
            assert dS_out.is_cuda and dS_out.dtype == torch.float64 and dS_out.stride(1) == 1
            sptr, lds = dS_out.data_ptr(), dS_out.stride(0)
        rc = load().concord_adjoint(self._ptr, gptr, gdt, ldg, float(tol), int(max_iter), sptr, lds,
                                    ctypes.byref(info))
        _check(rc, (OK, NOT_CONVERGED))
        return info

    def adjoint_data(self, X, prep: int = PREP_STANDARDIZE, dX_out=None):
        """dL/dX for the data X that S was computed from (after adjoint())."""
        import torch
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        if dX_out is None:
            dX_out = torch.empty(X.shape, dtype=X.dtype, device=X.device)
        _check(load().concord_adjoint_data(self._ptr, X.data_ptr(), _dtype_code(X), X.shape[0],
                                           X.stride(0), int(prep), dX_out.data_ptr(),
                                           _dtype_code(dX_out), dX_out.stride(0)))
        return dX_out

    def tune_lambda(self, S_val, lam0: float, steps: int = 20, lr: float = 0.5,
                    tol: float = 1e-5, max_sweeps: int = 1000, cg_tol: float = 1e-10):
        """Hypergradient descent on log lambda for the held-out loss; returns
        (steps, 6): lambda, loss, dL/dlambda, sweeps, CG iterations, KKT."""
        assert S_val.is_cuda and S_val.dim() == 2 and S_val.stride(1) == 1
        rows = np.zeros((int(steps), 6), dtype=np.float64)
        _check(load().concord_tune_lambda(self._ptr, S_val.data_ptr(), _dtype_code(S_val),
                                          S_val.stride(0), float(lam0), int(steps), float(lr),
                                          float(tol), int(max_sweeps), float(cg_tol),
                                          rows.ctypes.data_as(_dp)))
        return rows

    def solve_host(self, X: np.ndarray, lam: float, tol: float = 1e-5, max_sweeps: int = 1000,
                   prep: int = PREP_STANDARDIZE, stop_rule: int = STOP_KKT, Omega_out=None):
        assert X.dtype == np.float64 and X.flags.c_contiguous and X.shape[1] == self.p
        r = ConcordResult()
        optr = None
        if Omega_out is not None:
            assert Omega_out.dtype == np.float64 and Omega_out.flags.c_contiguous
            optr = Omega_out.ctypes.data_as(_dp)
        rc = load().concord_solve_host(self._ptr, X.ctypes.data_as(_dp), X.shape[0], int(prep),
                                       float(lam), float(tol), int(max_sweeps), int(stop_rule),
                                       optr, ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r


def concord_solve(data: np.ndarray, lam: float, tol: float = 1e-5, max_sweeps: int = 1000,
                  precision: int = FP64, is_X: bool = True, prep: int = PREP_STANDARDIZE,
                  Omega0: np.ndarray | None = None):
    """One-shot solve from host data; returns (Omega (p x p float64), ConcordResult)."""
    data = np.ascontiguousarray(data, dtype=np.float64)
    n, p = (data.shape if is_X else (0, data.shape[0]))
    Om = np.empty((p, p), dtype=np.float64)
    r = ConcordResult()
    o0 = None if Omega0 is None else np.ascontiguousarray(Omega0, dtype=np.float64)
    rc = load().concord_solve(data.ctypes.data_as(_dp), int(bool(is_X)), int(n), int(p),
                              int(prep), float(lam), float(tol), int(max_sweeps),
                              int(precision), o0.ctypes.data_as(_dp) if o0 is not None else None,
                              Om.ctypes.data_as(_dp), ctypes.byref(r))
    _check(rc, (OK, NOT_CONVERGED))
    return Om, r


# --------------------------------------------------------- joint estimator
class Joint:
    """Joint two-population CONCORD state (concord_joint_create): two
    precision matrices with lasso weight lambda1 and fusion weight lambda2."""

    def __init__(self, p: int, precision: int = FP64, device: int | None = None):
        import torch
        lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        self._ptr = ctypes.c_void_p()
        _check(lib.concord_joint_create(ctypes.byref(self._ptr), int(p), int(precision), dev))
        self.p, self.precision, self.device = int(p), int(precision), dev
        self.last = None

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            load().concord_joint_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream=None):
        _check(load().concord_joint_set_stream(self._ptr, _stream_ptr(stream)
                                               if stream is not False else None))

    def set_timeout(self, seconds: float):
        _check(load().concord_joint_set_timeout(self._ptr, float(seconds)))

    def set_grid(self, ctas: int):
        _check(load().concord_joint_set_grid(self._ptr, int(ctas)))

    def set_variant(self, variant: int):
        _check(load().concord_joint_set_variant(self._ptr, int(variant)))

    def set_fault(self, row: int, step: int = 0):
        """Failure testing: `row` skips publishing its version at colour step
        `step` of the next launch (concord_joint_set_fault)."""
        _check(load().concord_joint_set_fault(self._ptr, int(row), int(step)))

    def set_S(self, m: int, S):
        assert S.is_cuda and S.dim() == 2 and S.stride(1) == 1
        _check(load().concord_joint_set_S(self._ptr, int(m), S.data_ptr(), _dtype_code(S),
                                          S.stride(0)))

    def set_omega(self, m: int, Om):
        assert Om.is_cuda and Om.dim() == 2 and Om.stride(1) == 1
        _check(load().concord_joint_set_omega(self._ptr, int(m), Om.data_ptr(), _dtype_code(Om),
                                              Om.stride(0)))

    def get_omega(self, m: int, out=None):
        import torch
        if out is None:
            out = torch.empty((self.p, self.p), dtype=torch.float64,
                              device="cuda:%d" % self.device)
        assert out.is_cuda and out.stride(1) == 1
        _check(load().concord_joint_get_omega(self._ptr, int(m), out.data_ptr(), _dtype_code(out),
                                              out.stride(0)))
        return out

    def sweep(self, lam1: float, lam2: float, n_sweeps: int = 1) -> ConcordResult:
        r = ConcordResult()
        rc = load().concord_joint_sweep(self._ptr, float(lam1), float(lam2), int(n_sweeps),
                                        ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r

    def run(self, lam1: float, lam2: float, tol: float = 1e-5,
            max_sweeps: int = 1000) -> ConcordResult:
        r = ConcordResult()
        rc = load().concord_joint_run(self._ptr, float(lam1), float(lam2), float(tol),
                                      int(max_sweeps), ctypes.byref(r))
        self.last = r
        _check(rc, (OK, NOT_CONVERGED))
        return r

    def history(self) -> np.ndarray:
        """(rows, 4): delta, KKT residual, objective, pairs moved per sweep."""
        n = ctypes.c_int(0)
        _check(load().concord_joint_get_history(self._ptr, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 4), dtype=np.float64)
        if n.value:
            _check(load().concord_joint_get_history(self._ptr, out.ctypes.data_as(_dp), n.value,
                                                    ctypes.byref(n)))
        return out


# ------------------------------------------------- batched independent problems
class Batch:
    """Many independent CONCORD problems solved together (concord_batch_*):
    one persistent launch per wave of co-resident problems, each problem
    walking a warm-started lambda path."""

    def __init__(self, ps, precision: int = MIXED, n_cap: int = 0, device: int | None = None):
        import torch
        lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        ps = np.ascontiguousarray(ps, dtype=np.int32)
        self._ptr = ctypes.c_void_p()
        _check(lib.concord_batch_create(ctypes.byref(self._ptr), len(ps),
                                        ps.ctypes.data_as(_ip), int(precision), int(n_cap), dev))
        self.ps = [int(x) for x in ps]
        self.precision, self.n_cap, self.device = int(precision), int(n_cap), dev

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            load().concord_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __len__(self):
        return len(self.ps)

    def set_stream(self, stream=None):
        _check(load().concord_batch_set_stream(self._ptr, _stream_ptr(stream)
                                               if stream is not False else None))

    def set_timeout(self, seconds: float):
        _check(load().concord_batch_set_timeout(self._ptr, float(seconds)))

    def set_S(self, b: int, S):
        assert S.is_cuda and S.dim() == 2 and S.stride(1) == 1
        _check(load().concord_batch_set_S(self._ptr, int(b), S.data_ptr(), _dtype_code(S),
                                          S.stride(0)))

    def gram(self, b: int, X, rows=None, prep: int = PREP_STANDARDIZE):
        """S_b from the rows `rows` (CUDA int32 tensor, or None for all) of X."""
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        n = X.shape[0]
        if rows is not None:
            import torch
            assert rows.is_cuda and rows.dtype == torch.int32 and rows.dim() == 1
            rp, nr = rows.data_ptr(), rows.numel()
        else:
            rp, nr = None, n
        _check(load().concord_batch_gram(self._ptr, int(b), X.data_ptr(), _dtype_code(X), n,
                                         X.stride(0), rp, int(nr), int(prep)))

    def reset(self, b: int):
        _check(load().concord_batch_reset(self._ptr, int(b)))

    def set_rows_per_warp(self, rows: int):
        _check(load().concord_batch_set_rows_per_warp(self._ptr, int(rows)))

    def set_polish(self, on: bool):
        _check(load().concord_batch_set_polish(self._ptr, 1 if on else 0))

    def autotune(self, lam: float, sweeps: int = 2):
        ms = np.zeros(5, dtype=np.float64)
        _check(load().concord_batch_autotune(self._ptr, float(lam), int(sweeps),
                                             ms.ctypes.data_as(_dp)))
        return dict(zip((32, 16, 8, 4, 2), ms.tolist()))

    def info(self) -> dict:
        r, c, w = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        sec = ctypes.c_double(0.0)
        _check(load().concord_batch_info(self._ptr, ctypes.byref(r), ctypes.byref(c),
                                         ctypes.byref(w), ctypes.byref(sec)))
        return {"rows_per_warp": r.value, "ctas": c.value, "waves": w.value,
                "seconds": sec.value}

    def path(self, lambdas, tol: float = 1e-5, max_sweeps: int = 1000, support=None):
        """Returns res[b][k] (ConcordResult of problem b at lambda k)."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        B, K = len(self.ps), len(lam)
        res = (ConcordResult * (B * K))()
        sp = None
        if support is not None:
            import torch
            assert support.is_cuda and support.dtype == torch.float32
            assert support.numel() >= K * self.ps[0] * self.ps[0]
            sp = support.data_ptr()
        _check(load().concord_batch_path(self._ptr, lam.ctypes.data_as(_dp), K, float(tol),
                                         int(max_sweeps), res, sp))
        return [[res[b * K + k] for k in range(K)] for b in range(B)]

    def get_omega(self, b: int, dtype=None):
        import torch
        p = self.ps[b]
        out = torch.empty((p, p), dtype=dtype or torch.float64, device="cuda:%d" % self.device)
        _check(load().concord_batch_get_omega(self._ptr, int(b), out.data_ptr(), _dtype_code(out),
                                              out.stride(0)))
        return out
