"""CONCORD-PCD oracle (FP64, CPU): ctypes wrapper around ``concord_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It imports nothing
from the CUDA package and the CUDA package imports nothing from it.

Every function takes and returns float64 numpy arrays, row-major.  What each
one computes, and the passage of arXiv 2106.09382 it follows, is stated in the
C source beside it:

    standardize      Section 2.1 (X centered columnwise; unit 1/n variance)
    gram, gram_rows  Algorithm 1, T <- X^T X (here divided by n); selected rows
    eq3, eq2         Eq. 3 / Eq. 2 for one entry from explicit rows
    schedule         Section 3.2 circle method (round-robin table), colour order
    soft             Soft-threshold defined under Eq. 3
    offdiag_update   Eq. 3 with its two direct sums
    diag_update      Eq. 2 with its direct sum
    sweep            one outer iteration of Algorithm 1
    objective        Eq. 1 / n from S; objective_data: Eq. 1 / n from the data
    kkt              subgradient optimality conditions of Eq. 1
    solve            Algorithm 1 repeated until KKT <= tol
    solve_w, gram_w  the same solve with a maintained W = Omega S and the pairs
                     of a colour on OpenMP threads (Lemma 1), and the Gram on
                     threads: the timed CPU baseline (concord_oracle_w.c)
    joint_*          joint two-population CONCORD (the extension closing
                     Section 6): block update of (omega1_ij, omega2_ij) and of
                     the diagonal pair, sweep, objective, KKT, solve

``Oracle(path)`` binds any build of the same source (the planted-mistake
builds of the pin tests use it); the module-level functions use the normal
build.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "concord_oracle.c")
_SRC_W = os.path.join(_HERE, "concord_oracle_w.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_llp = ctypes.POINTER(ctypes.c_longlong)
_ci, _cd = ctypes.c_int, ctypes.c_double

_SIGNATURES = {
    "oracle_standardize": ([_dp, _ci, _ci, _ci, _dp], _ci),
    "oracle_gram": ([_dp, _ci, _ci, _dp], None),
    "oracle_gram_rows": ([_dp, _ci, _ci, _ip, _ci, _dp], None),
    "oracle_eq3": ([_dp, _dp, ctypes.c_size_t, _dp, _dp, _ci, _ci, _ci, _cd], _cd),
    "oracle_eq2": ([_dp, _dp, _ci, _ci], _cd),
    "oracle_schedule": ([_ci, _ip], _ci),
    "oracle_soft": ([_cd, _cd], _cd),
    "oracle_offdiag_update": ([_dp, _ci, _cd, _dp, _ci, _ci], _cd),
    "oracle_diag_update": ([_dp, _ci, _dp, _ci], _cd),
    "oracle_colour_steps": ([_dp, _ci, _cd, _dp, _ip, _ci, _ci, _ci, _llp], _cd),
    "oracle_diag_step": ([_dp, _ci, _dp], _cd),
    "oracle_sweep": ([_dp, _ci, _cd, _dp, _ip, _ci, _llp], _cd),
    "oracle_objective": ([_dp, _dp, _ci, _cd], _cd),
    "oracle_objective_data": ([_dp, _ci, _dp, _ci, _cd], _cd),
    "oracle_kkt": ([_dp, _dp, _ci, _cd], _cd),
    "oracle_solve": ([_dp, _ci, _cd, _cd, _cd, _ci, _dp, _dp, _dp, _dp], _ci),
    "oracle_joint_pair": ([_cd, _cd, _cd, _cd, _cd, _cd, _dp, _dp], None),
    "oracle_joint_diag": ([_cd, _cd, _cd, _cd, _cd, _dp, _dp], None),
    "oracle_joint_offdiag_update": ([_dp, _dp, _ci, _cd, _cd, _dp, _dp, _ci, _ci], _cd),
    "oracle_joint_diag_update": ([_dp, _dp, _ci, _cd, _dp, _dp, _ci], _cd),
    "oracle_joint_sweep": ([_dp, _dp, _ci, _cd, _cd, _dp, _dp, _ip, _ci, _llp], _cd),
    "oracle_joint_objective": ([_dp, _dp, _dp, _dp, _ci, _cd, _cd], _cd),
    "oracle_joint_kkt": ([_dp, _dp, _dp, _dp, _ci, _cd, _cd], _cd),
    "oracle_joint_solve": ([_dp, _dp, _ci, _cd, _cd, _cd, _cd, _ci, _dp, _dp, _dp, _dp, _dp,
                            _dp], _ci),
    "oracle_w_threads": ([_ci], _ci),
    "oracle_w_gram": ([_dp, _ci, _ci, _dp, _ci], _ci),
    "oracle_solve_w": ([_dp, _ci, _cd, _cd, _cd, _ci, _dp, _dp, _dp, _dp, _ci], _ci),
}


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle with gcc into ``oracle/_build/``.

    ``mutant`` > 0 builds planted mistake number ``mutant`` (pin tests only)
    into ``liboracle_mutant<k>.so``; 0 is the normal build ``liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB if mutant == 0 else os.path.join(_BUILD, "liboracle_mutant%d.so" % mutant)
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_W))):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           "-DORACLE_MUTANT=%d" % int(mutant), "-o", tmp, _SRC, _SRC_W, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def pe_of(p: int) -> int:
    """p rounded up to even (the paper's p_even)."""
    return p + (p % 2)


class Oracle:
    """One loaded build of ``concord_oracle.c``."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        self.lib = lib
        self.path = path

    def standardize(self, X, scale: bool = True) -> np.ndarray:
        X = _f64(X)
        n, p = X.shape
        Z = np.empty_like(X)
        rc = self.lib.oracle_standardize(_ptr(X), n, p, int(bool(scale)), _ptr(Z))
        if rc != 0:
            raise ValueError("oracle_standardize: constant column (status %d)" % rc)
        return Z

    def gram(self, Z) -> np.ndarray:
        Z = _f64(Z)
        n, p = Z.shape
        S = np.empty((p, p), dtype=np.float64)
        self.lib.oracle_gram(_ptr(Z), n, p, _ptr(S))
        return S

    def gram_rows(self, Z, rows) -> np.ndarray:
        """Rows `rows` of S = Z^T Z / n (same sums as gram)."""
        Z = _f64(Z)
        n, p = Z.shape
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rows.size, p), dtype=np.float64)
        self.lib.oracle_gram_rows(_ptr(Z), n, p, rows.ctypes.data_as(_ip), rows.size, _ptr(out))
        return out

    def eq3(self, om_row_i, om_col_j, s_row_i, s_row_j, i: int, j: int, lam: float) -> float:
        """Eq. 3 for pair (i, j) from row i and column j of Omega and rows i, j of S."""
        a, b = _f64(om_row_i), _f64(om_col_j)
        si, sj = _f64(s_row_i), _f64(s_row_j)
        return self.lib.oracle_eq3(_ptr(a), _ptr(b), 1, _ptr(si), _ptr(sj), a.size, int(i),
                                   int(j), float(lam))

    def eq2(self, om_row_i, s_row_i, i: int) -> float:
        """Eq. 2 for vertex i from row i of Omega and of S."""
        a, si = _f64(om_row_i), _f64(s_row_i)
        return self.lib.oracle_eq2(_ptr(a), _ptr(si), a.size, int(i))

    def schedule(self, p: int) -> np.ndarray:
        """(pe-1, pe/2, 2) int32 table of 0-based pairs; discarded pairs are -1."""
        pe = pe_of(p)
        pairs = np.empty((pe - 1, pe // 2, 2), dtype=np.int32)
        nc = self.lib.oracle_schedule(p, pairs.ctypes.data_as(_ip))
        if nc != pe - 1:
            raise ValueError("oracle_schedule failed (%d)" % nc)
        return pairs

    def soft(self, x: float, tau: float) -> float:
        return self.lib.oracle_soft(float(x), float(tau))

    def offdiag_update(self, S, Om: np.ndarray, lam: float, i: int, j: int) -> float:
        """Eq. 3 on (i, j); updates Om (float64, C-contiguous) in place."""
        S = _f64(S)
        assert Om.dtype == np.float64 and Om.flags.c_contiguous
        return self.lib.oracle_offdiag_update(_ptr(S), S.shape[0], float(lam), _ptr(Om), i, j)

    def diag_update(self, S, Om: np.ndarray, i: int) -> float:
        S = _f64(S)
        assert Om.dtype == np.float64 and Om.flags.c_contiguous
        return self.lib.oracle_diag_update(_ptr(S), S.shape[0], _ptr(Om), i)

    def colour_steps(self, S, Om: np.ndarray, lam: float, pairs: np.ndarray,
                     k_begin: int, k_end: int):
        """Colour steps k_begin..k_end-1 of `pairs` in place; (max |change|, #nonzero)."""
        S = _f64(S)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        nnz = ctypes.c_longlong(0)
        d = self.lib.oracle_colour_steps(_ptr(S), S.shape[0], float(lam), _ptr(Om),
                                         pairs.ctypes.data_as(_ip), pairs.shape[1],
                                         int(k_begin), int(k_end), ctypes.byref(nnz))
        return d, nnz.value

    def diag_step(self, S, Om: np.ndarray) -> float:
        S = _f64(S)
        return self.lib.oracle_diag_step(_ptr(S), S.shape[0], _ptr(Om))

    def sweep(self, S, Om: np.ndarray, lam: float, pairs: np.ndarray | None = None):
        """One Algorithm-1 iteration in place; returns (delta, #nonzero pair changes)."""
        S = _f64(S)
        p = S.shape[0]
        if pairs is None:
            pairs = self.schedule(p)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        nnz = ctypes.c_longlong(0)
        d = self.lib.oracle_sweep(_ptr(S), p, float(lam), _ptr(Om),
                                  pairs.ctypes.data_as(_ip), pairs.shape[0], ctypes.byref(nnz))
        return d, nnz.value

    def objective(self, S, Om, lam: float) -> float:
        S, Om = _f64(S), _f64(Om)
        return self.lib.oracle_objective(_ptr(S), _ptr(Om), S.shape[0], float(lam))

    def objective_data(self, Z, Om, lam: float) -> float:
        Z, Om = _f64(Z), _f64(Om)
        n, p = Z.shape
        return self.lib.oracle_objective_data(_ptr(Z), n, _ptr(Om), p, float(lam))

    def kkt(self, S, Om, lam: float) -> float:
        S, Om = _f64(S), _f64(Om)
        return self.lib.oracle_kkt(_ptr(S), _ptr(Om), S.shape[0], float(lam))

    def solve(self, S, lam: float, tol: float = 1e-5, max_sweeps: int = 1000, Om0=None,
              delta_tol: float = 1e-5, history: bool = False):
        """Algorithm 1 until KKT <= tol.  Returns (Omega, info dict)."""
        S = _f64(S)
        p = S.shape[0]
        Om = np.empty((p, p), dtype=np.float64)
        stats = np.zeros(6, dtype=np.float64)
        hist = np.zeros((max(max_sweeps, 1), 3), dtype=np.float64) if history else None
        o0 = _f64(Om0) if Om0 is not None else None
        rc = self.lib.oracle_solve(_ptr(S), p, float(lam), float(tol), float(delta_tol),
                                   int(max_sweeps), _ptr(o0) if o0 is not None else None,
                                   _ptr(Om), _ptr(stats),
                                   _ptr(hist) if hist is not None else None)
        if rc < 0:
            raise ValueError("oracle_solve: status %d" % rc)
        info = dict(converged=(rc == 0), sweeps=int(stats[0]), objective=float(stats[1]),
                    kkt=float(stats[2]), delta=float(stats[3]),
                    first_delta_sweep=int(stats[4]), nonzero_changes=int(stats[5]))
        if hist is not None:
            info["history"] = hist[: info["sweeps"]].copy()
        return Om, info

    # ------------------------------------------------ maintained-product mode
    def threads(self, threads: int = 0) -> int:
        """Threads the maintained-product mode runs with (0 = all cores)."""
        return int(self.lib.oracle_w_threads(int(threads)))

    def gram_w(self, Z, threads: int = 0) -> np.ndarray:
        """S = Z^T Z / n on host threads (upper triangle, k ascending, mirrored)."""
        Z = _f64(Z)
        n, p = Z.shape
        S = np.empty((p, p), dtype=np.float64)
        if self.lib.oracle_w_gram(_ptr(Z), n, p, _ptr(S), int(threads)) != 0:
            raise ValueError("oracle_w_gram: bad arguments")
        return S

    def solve_w(self, S, lam: float, tol: float = 1e-5, max_sweeps: int = 1000, Om0=None,
                delta_tol: float = 1e-5, history: bool = False, threads: int = 0):
        """The solve of `solve` with a maintained W = Omega S and the pairs of
        each colour (and the diagonal updates) spread over host threads.
        Returns (Omega, info dict) like `solve`, plus info["threads"]."""
        S = _f64(S)
        p = S.shape[0]
        Om = np.empty((p, p), dtype=np.float64)
        stats = np.zeros(7, dtype=np.float64)
        hist = np.zeros((max(max_sweeps, 1), 3), dtype=np.float64) if history else None
        o0 = _f64(Om0) if Om0 is not None else None
        rc = self.lib.oracle_solve_w(_ptr(S), p, float(lam), float(tol), float(delta_tol),
                                     int(max_sweeps), _ptr(o0) if o0 is not None else None,
                                     _ptr(Om), _ptr(stats),
                                     _ptr(hist) if hist is not None else None, int(threads))
        if rc < 0:
            raise ValueError("oracle_solve_w: status %d" % rc)
        info = dict(converged=(rc == 0), sweeps=int(stats[0]), objective=float(stats[1]),
                    kkt=float(stats[2]), delta=float(stats[3]),
                    first_delta_sweep=int(stats[4]), nonzero_changes=int(stats[5]),
                    threads=int(stats[6]))
        if hist is not None:
            info["history"] = hist[: info["sweeps"]].copy()
        return Om, info

    # ---- joint two-population CONCORD
    def joint_pair(self, c1, g1, c2, g2, l1, l2):
        """Minimiser (x, y) of the two-variable block problem of the joint
        objective (see oracle_joint_pair)."""
        x, y = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_joint_pair(float(c1), float(g1), float(c2), float(g2), float(l1),
                                   float(l2), ctypes.byref(x), ctypes.byref(y))
        return x.value, y.value

    def joint_diag(self, s1, b1, s2, b2, l2):
        """Minimiser (d1, d2) of the diagonal block problem."""
        x, y = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_joint_diag(float(s1), float(b1), float(s2), float(b2), float(l2),
                                   ctypes.byref(x), ctypes.byref(y))
        return x.value, y.value

    def joint_offdiag_update(self, S1, S2, Om1, Om2, l1, l2, i, j) -> float:
        S1, S2 = _f64(S1), _f64(S2)
        for Om in (Om1, Om2):
            assert Om.dtype == np.float64 and Om.flags.c_contiguous
        return self.lib.oracle_joint_offdiag_update(_ptr(S1), _ptr(S2), S1.shape[0], float(l1),
                                                    float(l2), _ptr(Om1), _ptr(Om2), int(i),
                                                    int(j))

    def joint_diag_update(self, S1, S2, Om1, Om2, l2, i) -> float:
        S1, S2 = _f64(S1), _f64(S2)
        return self.lib.oracle_joint_diag_update(_ptr(S1), _ptr(S2), S1.shape[0], float(l2),
                                                 _ptr(Om1), _ptr(Om2), int(i))

    def joint_sweep(self, S1, S2, Om1, Om2, l1, l2, pairs=None):
        """One joint sweep in place; returns (delta, #pairs that moved)."""
        S1, S2 = _f64(S1), _f64(S2)
        p = S1.shape[0]
        if pairs is None:
            pairs = self.schedule(p)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        nnz = ctypes.c_longlong(0)
        d = self.lib.oracle_joint_sweep(_ptr(S1), _ptr(S2), p, float(l1), float(l2), _ptr(Om1),
                                        _ptr(Om2), pairs.ctypes.data_as(_ip), pairs.shape[0],
                                        ctypes.byref(nnz))
        return d, nnz.value

    def joint_objective(self, S1, S2, Om1, Om2, l1, l2) -> float:
        S1, S2, Om1, Om2 = _f64(S1), _f64(S2), _f64(Om1), _f64(Om2)
        return self.lib.oracle_joint_objective(_ptr(S1), _ptr(S2), _ptr(Om1), _ptr(Om2),
                                               S1.shape[0], float(l1), float(l2))

    def joint_kkt(self, S1, S2, Om1, Om2, l1, l2) -> float:
        S1, S2, Om1, Om2 = _f64(S1), _f64(S2), _f64(Om1), _f64(Om2)
        return self.lib.oracle_joint_kkt(_ptr(S1), _ptr(S2), _ptr(Om1), _ptr(Om2), S1.shape[0],
                                         float(l1), float(l2))

    def joint_solve(self, S1, S2, l1, l2, tol=1e-5, max_sweeps=1000, Om0=None,
                    delta_tol=1e-5, history=False):
        """Joint sweeps until the joint KKT residual <= tol.  Returns
        (Omega1, Omega2, info dict); Om0 is None or a pair of starting points."""
        S1, S2 = _f64(S1), _f64(S2)
        p = S1.shape[0]
        Om1 = np.empty((p, p), dtype=np.float64)
        Om2 = np.empty((p, p), dtype=np.float64)
        stats = np.zeros(6, dtype=np.float64)
        hist = np.zeros((max(max_sweeps, 1), 3), dtype=np.float64) if history else None
        i1 = _f64(Om0[0]) if Om0 is not None else None
        i2 = _f64(Om0[1]) if Om0 is not None else None
        rc = self.lib.oracle_joint_solve(_ptr(S1), _ptr(S2), p, float(l1), float(l2), float(tol),
                                         float(delta_tol), int(max_sweeps),
                                         _ptr(i1) if i1 is not None else None,
                                         _ptr(i2) if i2 is not None else None,
                                         _ptr(Om1), _ptr(Om2), _ptr(stats),
                                         _ptr(hist) if hist is not None else None)
        if rc < 0:
            raise ValueError("oracle_joint_solve: status %d" % rc)
        info = dict(converged=(rc == 0), sweeps=int(stats[0]), objective=float(stats[1]),
                    kkt=float(stats[2]), delta=float(stats[3]),
                    first_delta_sweep=int(stats[4]), nonzero_changes=int(stats[5]))
        if hist is not None:
            info["history"] = hist[: info["sweeps"]].copy()
        return Om1, Om2, info


_lock = threading.Lock()
_default: Oracle | None = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def load_mutant(k: int) -> Oracle:
    """A build carrying planted mistake k (pin tests only)."""
    return Oracle(build(mutant=k))


def standardize(X, scale: bool = True):
    return default().standardize(X, scale)


def gram(Z):
    return default().gram(Z)


def schedule(p: int):
    return default().schedule(p)


def gram_rows(Z, rows):
    return default().gram_rows(Z, rows)


def eq3(om_row_i, om_col_j, s_row_i, s_row_j, i, j, lam):
    return default().eq3(om_row_i, om_col_j, s_row_i, s_row_j, i, j, lam)


def eq2(om_row_i, s_row_i, i):
    return default().eq2(om_row_i, s_row_i, i)


def soft(x, tau):
    return default().soft(x, tau)


def offdiag_update(S, Om, lam, i, j):
    return default().offdiag_update(S, Om, lam, i, j)


def diag_update(S, Om, i):
    return default().diag_update(S, Om, i)


def colour_steps(S, Om, lam, pairs, k_begin, k_end):
    return default().colour_steps(S, Om, lam, pairs, k_begin, k_end)


def diag_step(S, Om):
    return default().diag_step(S, Om)


def sweep(S, Om, lam, pairs=None):
    return default().sweep(S, Om, lam, pairs)


def objective(S, Om, lam):
    return default().objective(S, Om, lam)


def objective_data(Z, Om, lam):
    return default().objective_data(Z, Om, lam)


def kkt(S, Om, lam):
    return default().kkt(S, Om, lam)


def solve(S, lam, tol=1e-5, max_sweeps=1000, Om0=None, delta_tol=1e-5, history=False):
    return default().solve(S, lam, tol, max_sweeps, Om0, delta_tol, history)


def threads(n: int = 0) -> int:
    return default().threads(n)


def gram_w(Z, threads: int = 0):
    return default().gram_w(Z, threads)


def solve_w(S, lam, tol=1e-5, max_sweeps=1000, Om0=None, delta_tol=1e-5, history=False,
            threads=0):
    return default().solve_w(S, lam, tol, max_sweeps, Om0, delta_tol, history, threads)


def lambda_max(S) -> float:
    """Smallest lambda at which the diagonal point diag(s_ii^{-1/2}) is optimal:
    max_{i<j} |s_ij| (s_ii^{-1/2} + s_jj^{-1/2}), from the KKT conditions of
    Eq. 1 at a diagonal Omega, where G_ij = s_ij (omega_ii + omega_jj)."""
    S = _f64(S)
    r = 1.0 / np.sqrt(np.diag(S))
    M = np.abs(S) * (r[:, None] + r[None, :])
    np.fill_diagonal(M, 0.0)
    return float(M.max())


def joint_pair(c1, g1, c2, g2, l1, l2):
    return default().joint_pair(c1, g1, c2, g2, l1, l2)


def joint_diag(s1, b1, s2, b2, l2):
    return default().joint_diag(s1, b1, s2, b2, l2)


def joint_sweep(S1, S2, Om1, Om2, l1, l2, pairs=None):
    return default().joint_sweep(S1, S2, Om1, Om2, l1, l2, pairs)


def joint_objective(S1, S2, Om1, Om2, l1, l2):
    return default().joint_objective(S1, S2, Om1, Om2, l1, l2)


def joint_kkt(S1, S2, Om1, Om2, l1, l2):
    return default().joint_kkt(S1, S2, Om1, Om2, l1, l2)


def joint_solve(S1, S2, l1, l2, tol=1e-5, max_sweeps=1000, Om0=None, delta_tol=1e-5,
                history=False):
    return default().joint_solve(S1, S2, l1, l2, tol, max_sweeps, Om0, delta_tol, history)
