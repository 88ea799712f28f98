"""Plain FP64 CPU oracle for the inverse-factorization path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library's
compute path never loads it, and it shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C loops, FP64).  This module only
marshals numpy arrays in and out.  Functions, each following the paper
(Artemov, Rudberg, Rubensson, arXiv:1901.07993):

* ``truncate``   -- block removal when ||block||_F < tau (Section 5).
* ``gemm``       -- alpha op(A) op(B) on stored blocks, then truncation of the
                    output blocks (Section 5, truncation after every product).
* ``add``        -- alpha A + beta B + gamma I on the union pattern.
* ``gershgorin`` -- beta = max_i sum_j |S_ij| (Section 2.2).
* ``irsi``       -- refinement from Z_0 = c I, Eq. (2.1), direct delta, the
                    automatic stop rule of Section 2.2.
* ``lif``        -- localized inverse factorization, Algorithm 2 with the
                    localized update of Eq. (2.2) and the stop of Algorithm 4.
* ``invchol``    -- leaf routine: S = L L^T, Z = L^-T.
* ``resid``      -- ||I - Z^T S Z||_F with untruncated products.

Pins (tests/test_oracle_*.py) tie each function to the mathematics:
brute-force dense products, the closed-form eigenvalue recurrence of the
refinement from a scaled identity, S^-1/2 by eigendecomposition, the LIF fixed
point Z_0 (Z_0^T S Z_0)^-1/2, library Cholesky, and Z^T S Z = I.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

STOP_RULE, STOP_TARGET, STOP_MAXITER, STOP_FIXED = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O3", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        # OpenMP over output block rows where the compiler has it; plain otherwise
        if subprocess.call(base[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel block-row loop (1 = single-threaded)."""
    _load().om_set_threads(int(n))


def max_threads() -> int:
    """Threads the parallel loop uses now (1 in a build without OpenMP)."""
    return int(_load().om_max_threads())


class _Opts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("tau", ctypes.c_double), ("target", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("fixed_iters", ctypes.c_int),
                ("c_rule", ctypes.c_int), ("leaf_size", ctypes.c_int), ("rinch_rows", ctypes.c_int),
                ("local_delta", ctypes.c_int)]


class _Rep(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("stop_reason", ctypes.c_int), ("levels", ctypes.c_int),
                ("beta", ctypes.c_double), ("delta_fro", ctypes.c_double * 64),
                ("n_delta", ctypes.c_int), ("products", ctypes.c_int64),
                ("block_pairs", ctypes.c_int64), ("status", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "om_from_arrays": ([i64, i32, i32, i64, p, p, p], p),
            "om_free": ([p], None),
            "om_nnzb": ([p], i64),
            "om_nb": ([p], i32),
            "om_n": ([p], i64),
            "om_to_arrays": ([p, p, p, p], None),
            "om_truncate": ([p, d], p),
            "om_transpose": ([p], p),
            "om_gemm": ([p, i32, p, i32, d, d], p),
            "om_add": ([d, p, d, p, d], p),
            "om_fro": ([p], d),
            "om_gershgorin": ([p], d),
            "om_coef_b": ([i32], d),
            "om_irsi": ([p, ctypes.POINTER(_Opts), ctypes.POINTER(_Rep)], p),
            "om_lif": ([p, ctypes.POINTER(_Opts), ctypes.POINTER(_Rep)], p),
            "om_rinch": ([p, ctypes.POINTER(_Opts), ctypes.POINTER(_Rep)], p),
            "om_invchol_dense": ([i32, p, p], i32),
            "om_resid": ([p, p], d),
            "om_counter_products": ([], i64),
            "om_counter_pairs": ([], i64),
            "om_set_threads": ([i32], None),
            "om_max_threads": ([], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


@dataclass
class Mat:
    """Oracle-side block-sparse matrix (host numpy arrays, FP64)."""
    n: int
    bs: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray  # [nnzb, bs, bs]

    @property
    def nb(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnzb(self) -> int:
        return len(self.col_idx)

    def to_dense(self) -> np.ndarray:
        nb, bs = self.nb, self.bs
        d = np.zeros((nb * bs, nb * bs))
        rows = np.repeat(np.arange(nb), np.diff(self.row_ptr))
        for p, (i, j) in enumerate(zip(rows, self.col_idx)):
            d[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = self.val[p]
        return d

    def blocks(self) -> dict:
        rows = np.repeat(np.arange(self.nb), np.diff(self.row_ptr))
        return {(int(i), int(j)): self.val[p] for p, (i, j) in enumerate(zip(rows, self.col_idx))}


def _to_c(a) -> int:
    lib = _load()
    rp = np.ascontiguousarray(a.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(a.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(a.val, dtype=np.float64)
    h = lib.om_from_arrays(int(a.n), int(a.bs), len(rp) - 1, len(ci),
                           rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    return h


def _from_c(h, bs: int) -> Mat:
    lib = _load()
    nb, nnzb, n = lib.om_nb(h), lib.om_nnzb(h), lib.om_n(h)
    rp = np.zeros(nb + 1, dtype=np.int32)
    ci = np.zeros(nnzb, dtype=np.int32)
    v = np.zeros((nnzb, bs, bs))
    lib.om_to_arrays(h, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    lib.om_free(h)
    return Mat(int(n), bs, rp, ci, v)


class _Held:
    """C handles freed on exit."""

    def __init__(self, *mats):
        self.h = [_to_c(m) if m is not None else None for m in mats]

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        for h in self.h:
            if h:
                _load().om_free(h)


def from_dense(d: np.ndarray, bs: int, n: int | None = None, keep_zero: bool = False) -> Mat:
    """Block a dense matrix; all-zero blocks are not stored unless keep_zero."""
    N = d.shape[0]
    nb = N // bs
    rp, ci, vals = [0], [], []
    for i in range(nb):
        for j in range(nb):
            blk = d[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]
            if keep_zero or np.any(blk != 0):
                ci.append(j)
                vals.append(blk.copy())
        rp.append(len(ci))
    v = np.array(vals) if vals else np.zeros((0, bs, bs))
    return Mat(n if n is not None else N, bs, np.array(rp, np.int32), np.array(ci, np.int32), v)


def truncate(a, tau: float) -> Mat:
    with _Held(a) as (h,):
        return _from_c(_load().om_truncate(h, tau), a.bs)


def transpose(a) -> Mat:
    with _Held(a) as (h,):
        return _from_c(_load().om_transpose(h), a.bs)


def gemm(a, b, trans_a: bool = False, trans_b: bool = False, alpha: float = 1.0, tau: float = 0.0) -> Mat:
    with _Held(a, b) as (ha, hb):
        return _from_c(_load().om_gemm(ha, int(trans_a), hb, int(trans_b), alpha, tau), a.bs)


def add(alpha: float, a, beta: float = 0.0, b=None, gamma: float = 0.0) -> Mat:
    with _Held(a, b) as (ha, hb):
        return _from_c(_load().om_add(alpha, ha, beta, hb, gamma), a.bs)


def fro(a) -> float:
    with _Held(a) as (h,):
        return float(_load().om_fro(h))


def gershgorin(a) -> float:
    with _Held(a) as (h,):
        return float(_load().om_gershgorin(h))


def coef_b(k: int) -> float:
    return float(_load().om_coef_b(k))


@dataclass
class Report:
    sweeps: int
    stop_reason: int
    levels: int
    beta: float
    delta_fro: list = field(default_factory=list)
    products: int = 0
    block_pairs: int = 0
    status: int = 0


def _opts(m, tau, target, max_iter, fixed_iters, c_rule, leaf_size, rinch_rows=0, local_delta=0) -> _Opts:
    return _Opts(m, tau, target, max_iter, fixed_iters, c_rule, leaf_size, rinch_rows, local_delta)


def _report(r: _Rep) -> Report:
    return Report(r.sweeps, r.stop_reason, r.levels, r.beta, [r.delta_fro[i] for i in range(r.n_delta)],
                  r.products, r.block_pairs, r.status)


def irsi(S, m: int = 2, tau: float = 1e-10, target: float = 0.0, max_iter: int = 50,
         fixed_iters: int = 0, c_rule: int = 0, local_delta: bool = False):
    """Iterative refinement from Z_0 = c I (Eq. 2.1): direct delta each sweep,
    or the local update of Eq. (2.2) after a direct delta_0. Returns (Z, Report)."""
    o = _opts(m, tau, target, max_iter, fixed_iters, c_rule, 0, 0, int(local_delta))
    r = _Rep()
    with _Held(S) as (h,):
        z = _load().om_irsi(h, ctypes.byref(o), ctypes.byref(r))
    return _from_c(z, S.bs), _report(r)


def lif(S, m: int = 2, tau: float = 1e-10, target: float = 0.0, max_iter: int = 50, leaf_size: int = 512,
        rinch_rows: int = 0):
    """Localized inverse factorization (Algorithm 2); sub-problems with at most
    rinch_rows rows (when above leaf_size) are factorized by RINCH. Returns (Z, Report)."""
    o = _opts(m, tau, target, max_iter, 0, 0, leaf_size, rinch_rows)
    r = _Rep()
    with _Held(S) as (h,):
        z = _load().om_lif(h, ctypes.byref(o), ctypes.byref(r))
    return _from_c(z, S.bs), _report(r)


def rinch(S, tau: float = 1e-10, leaf_size: int = 512):
    """Recursive inverse Cholesky (Algorithm 1) with the dense leaf routine
    below leaf_size rows.  Returns (Z, Report); Report.levels = recursion depth."""
    o = _opts(2, tau, 0.0, 50, 0, 0, leaf_size)
    r = _Rep()
    with _Held(S) as (h,):
        z = _load().om_rinch(h, ctypes.byref(o), ctypes.byref(r))
    return _from_c(z, S.bs), _report(r)


def invchol(S: np.ndarray) -> np.ndarray:
    """Dense leaf routine: Z = L^-T for S = L L^T.  Raises if S is not SPD."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    n = S.shape[0]
    Z = np.zeros_like(S)
    rc = _load().om_invchol_dense(n, S.ctypes.data, Z.ctypes.data)
    if rc != 0:
        raise np.linalg.LinAlgError("leaf matrix not positive definite")
    return Z


def resid(S, Z) -> float:
    """||I - Z^T S Z||_F with untruncated products."""
    with _Held(S, Z) as (hs, hz):
        return float(_load().om_resid(hs, hz))


# ---------------------------------------------------------------------------
# adjoint of the refinement on a frozen block pattern
# ---------------------------------------------------------------------------
def _load_adjoint():
    lib = _load()
    if not hasattr(lib, "_adj_ready"):
        p, i32, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "om_tape_record": ([p, d, i32, d], p),
            "om_tape_free": ([p], None),
            "om_frozen_loss": ([p, p, p, d], d),
            "om_adjoint": ([p, p], p),
            "om_tape_loss": ([p, p], d),
            "om_tape_S": ([p], p),
            "om_tape_Z": ([p, i32], p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        lib._adj_ready = True
    return lib


def _copy_borrowed(h, bs: int) -> Mat:
    lib = _load()
    nb, nnzb, n = lib.om_nb(h), lib.om_nnzb(h), lib.om_n(h)
    rp = np.zeros(nb + 1, dtype=np.int32)
    ci = np.zeros(nnzb, dtype=np.int32)
    v = np.zeros((nnzb, bs, bs))
    lib.om_to_arrays(h, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    return Mat(int(n), bs, rp, ci, v)


class Tape:
    """Recording run of K truncated sweeps (m = 2) from Z_0 = c I; its block
    patterns are the frozen patterns of the differentiated function."""

    def __init__(self, S, c: float, K: int, tau: float):
        lib = _load_adjoint()
        self.bs, self.c, self.K = S.bs, c, K
        with _Held(S) as (hs,):
            self.h = lib.om_tape_record(hs, c, K, tau)

    def S(self) -> Mat:
        return _copy_borrowed(_load_adjoint().om_tape_S(self.h), self.bs)

    def Z(self, k: int) -> Mat:
        return _copy_borrowed(_load_adjoint().om_tape_Z(self.h, k), self.bs)

    def loss(self, F) -> float:
        with _Held(F) as (hf,):
            return float(_load_adjoint().om_tape_loss(self.h, hf))

    def frozen_loss(self, S, F) -> float:
        """L for another S on the frozen patterns (S must have the tape's S pattern)."""
        with _Held(S, F) as (hs, hf):
            return float(_load_adjoint().om_frozen_loss(self.h, hs, hf, self.c))

    def adjoint(self, F) -> Mat:
        """dL/dS (all entries independent) on the pattern of the truncated S."""
        with _Held(F) as (hf,):
            return _from_c(_load_adjoint().om_adjoint(self.h, hf), self.bs)

    def __del__(self):
        try:
            if self.h:
                _load_adjoint().om_tape_free(self.h)
        except Exception:
            pass
