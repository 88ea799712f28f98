"""Python binding of the C ABI in include/ifac.h (argument marshalling only).

Every computation runs in libifac.so's CUDA kernels; this module converts
arguments, owns the returned device matrices (freed with ifac_bsr_free) and
raises IfacError on negative status codes.  It never falls back to another
implementation: if the library is missing, loading raises.

Function names follow the C ABI: bsr_gemm_trunc, bsr_gemm_sym_trunc, bsr_add,
bsr_truncate, bsr_fro, bsr_gershgorin, leaf_invchol_batched,
inv_factor_refine, inv_factor_localized, inv_factor_rinch, inv_factor_resid.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libifac.so")

OK, WARN_TARGET_NOT_MET = 0, 1
TF32, BF16, FP64_SPLIT = 1, 2, 3
ERR_INVALID, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -7
ERR_TIMEOUT, ERR_TOO_LARGE = -6, -8
FP64 = 0
STOP_RULE, STOP_TARGET, STOP_MAXITER, STOP_FIXED = 1, 2, 3, 4

EXPORTS = ("ifac_create", "ifac_destroy", "ifac_set_stream", "ifac_last_error", "ifac_opts_default",
           "ifac_bsr_upload", "ifac_bsr_download", "ifac_bsr_free", "bsr_gemm_trunc", "bsr_gemm_sym_trunc",
           "bsr_add", "bsr_truncate", "bsr_fro", "bsr_gershgorin", "leaf_invchol_batched", "inv_factor_refine",
           "inv_factor_localized", "inv_factor_resid", "leaf_invchol_batched_noalloc",
           "inv_factor_refine_adjoint", "inv_factor_refine_batched", "ifac_set_split_slices",
           "inv_factor_rinch", "ifac_selftest_wait_timeout", "bsr_reblock", "ifac_set_schedule",
           "ifac_autotune_batched", "ifac_set_fp32_intermediates")


class IfacError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ifac error {code}: {msg}")
        self.code = code


class _Bsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("bs", ctypes.c_int32), ("nb", ctypes.c_int32), ("nnzb", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("norms", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("max_iter", ctypes.c_int), ("fixed_iters", ctypes.c_int),
                ("c_rule", ctypes.c_int), ("leaf_size", ctypes.c_int), ("prec", ctypes.c_int),
                ("profile", ctypes.c_int), ("delta_prec", ctypes.c_int), ("rinch_rows", ctypes.c_int),
                ("local_delta", ctypes.c_int)]


class _Report(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("stop_reason", ctypes.c_int), ("levels", ctypes.c_int),
                ("n_delta", ctypes.c_int), ("beta", ctypes.c_double), ("delta_fro", ctypes.c_double * 64),
                ("products", ctypes.c_int64), ("block_pairs", ctypes.c_int64), ("nnzb_Z", ctypes.c_int64),
                ("flops", ctypes.c_double), ("fp64_delta_evals", ctypes.c_int), ("low_sweeps", ctypes.c_int),
                ("launches", ctypes.c_int64), ("gemm_launches", ctypes.c_int64), ("gemm_ms", ctypes.c_double),
                ("fp64_pairs", ctypes.c_int64), ("tc_launches", ctypes.c_int64), ("tc_ms", ctypes.c_double),
                ("tc_pairs", ctypes.c_int64), ("resid_fro", ctypes.c_double), ("split_launches", ctypes.c_int64),
                ("split_ms", ctypes.c_double), ("split_pairs", ctypes.c_int64),
                ("split_slice_pairs", ctypes.c_int64), ("fp64_bytes", ctypes.c_double),
                ("tc_bytes", ctypes.c_double), ("split_bytes", ctypes.c_double)]


class _TuneResult(ctypes.Structure):
    _fields_ = [("bs", ctypes.c_int32), ("narrow_kmax", ctypes.c_int32), ("narrow_kmax_split", ctypes.c_int32),
                ("low_sweeps_est", ctypes.c_int32), ("split_evals_est", ctypes.c_int32),
                ("probe_ms", ctypes.c_double * 3), ("probe64_lp_ms", ctypes.c_double * 3),
                ("probe64_split_ms", ctypes.c_double * 3)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libifac.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    p, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PB = ctypes.POINTER(_Bsr)
    sig = {
        "ifac_create": ([ctypes.POINTER(p), p, p], i32),
        "ifac_destroy": ([p], None),
        "ifac_set_stream": ([p, p], i32),
        "ifac_set_split_slices": ([p, i32], i32),
        "ifac_set_fp32_intermediates": ([p, i32], i32),
        "ifac_last_error": ([p], ctypes.c_char_p),
        "ifac_opts_default": ([ctypes.POINTER(_Opts)], None),
        "ifac_bsr_upload": ([p, i64, i32, i32, i64, p, p, p, PB], i32),
        "ifac_bsr_download": ([p, PB, p, p, p], i32),
        "ifac_bsr_free": ([p, PB], None),
        "bsr_gemm_trunc": ([p, PB, i32, PB, i32, d, d, i32, PB], i32),
        "bsr_gemm_sym_trunc": ([p, PB, i32, PB, i32, d, d, i32, PB], i32),
        "bsr_add": ([p, d, PB, d, PB, d, PB], i32),
        "bsr_truncate": ([p, PB, d, PB], i32),
        "bsr_fro": ([p, PB, ctypes.POINTER(d)], i32),
        "bsr_gershgorin": ([p, PB, ctypes.POINTER(d)], i32),
        "leaf_invchol_batched": ([p, i32, i32, p, p, p], i32),
        "inv_factor_refine": ([p, PB, d, d, ctypes.POINTER(_Opts), PB, ctypes.POINTER(_Report)], i32),
        "inv_factor_localized": ([p, PB, d, d, ctypes.POINTER(_Opts), PB, ctypes.POINTER(_Report)], i32),
        "inv_factor_rinch": ([p, PB, d, ctypes.POINTER(_Opts), PB, ctypes.POINTER(_Report)], i32),
        "inv_factor_resid": ([p, PB, PB, ctypes.POINTER(d)], i32),
        "leaf_invchol_batched_noalloc": ([p, i32, i32, p, p, p], i32),
        "inv_factor_refine_adjoint": ([p, PB, PB, i32, d, ctypes.POINTER(d), PB], i32),
        "inv_factor_refine_batched": ([p, i32, p, d, d, ctypes.POINTER(_Opts), p, p], i32),
        "ifac_selftest_wait_timeout": ([p, i64], i32),
        "bsr_reblock": ([p, PB, i32, PB], i32),
        "ifac_set_schedule": ([p, i32, i32], i32),
        "ifac_autotune_batched": ([p, i32, p, d, ctypes.POINTER(_Opts), ctypes.POINTER(_TuneResult)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


class Context:
    """A library context on the current device and (by default) torch's current stream.

    allocator: optional (alloc, free) pair of Python callables, alloc(bytes,
    stream) -> device address or 0 on failure, free(address, stream); the
    library then takes every device buffer from it (ifac_allocator)."""

    def __init__(self, stream: int | None = None, allocator=None):
        self.lib = load()
        h = ctypes.c_void_p()
        arg = None
        if allocator is not None:
            a_fn, f_fn = allocator
            # the callbacks must outlive the context
            self._alloc_cb = _ALLOC_FN(lambda user, nbytes, st: a_fn(int(nbytes), st or 0) or None)
            self._free_cb = _FREE_FN(lambda user, ptr, st: f_fn(ptr, st or 0))
            self._alloc = _Allocator(self._alloc_cb, self._free_cb, None)
            arg = ctypes.byref(self._alloc)
        rc = self.lib.ifac_create(ctypes.byref(h), ctypes.c_void_p(_current_stream() if stream is None else stream),
                                  arg)
        if rc != 0:
            raise IfacError(rc, "ifac_create failed")
        self.h = h

    def check(self, rc: int) -> int:
        if rc < 0:
            raise IfacError(rc, self.lib.ifac_last_error(self.h).decode())
        return rc

    def set_stream(self, stream: int):
        self.check(self.lib.ifac_set_stream(self.h, ctypes.c_void_p(stream)))

    def set_split_slices(self, slices: int):
        self.check(self.lib.ifac_set_split_slices(self.h, int(slices)))

    def set_fp32_intermediates(self, on: bool):
        self.check(self.lib.ifac_set_fp32_intermediates(self.h, 1 if on else 0))

    def close(self):
        if getattr(self, "h", None):
            self.lib.ifac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceBSR:
    """A library-allocated device matrix (freed when garbage-collected)."""

    def __init__(self, ctx: Context, raw: _Bsr):
        self.ctx = ctx
        self.raw = raw

    n = property(lambda self: int(self.raw.n))
    bs = property(lambda self: int(self.raw.bs))
    nb = property(lambda self: int(self.raw.nb))
    nnzb = property(lambda self: int(self.raw.nnzb))

    def ptr(self):
        return ctypes.byref(self.raw)

    def download(self) -> "HostMatrix":
        rp = np.zeros(self.nb + 1, dtype=np.int32)
        ci = np.zeros(self.nnzb, dtype=np.int32)
        v = np.zeros((self.nnzb, self.bs, self.bs))
        self.ctx.check(self.ctx.lib.ifac_bsr_download(self.ctx.h, self.ptr(), rp.ctypes.data, ci.ctypes.data,
                                                      v.ctypes.data))
        return HostMatrix(self.n, self.bs, rp, ci, v)

    def free(self):
        if self.raw is not None and self.ctx.h:
            self.ctx.lib.ifac_bsr_free(self.ctx.h, ctypes.byref(self.raw))
        self.raw = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


@dataclass
class HostMatrix:
    n: int
    bs: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nb(self):
        return len(self.row_ptr) - 1

    @property
    def nnzb(self):
        return len(self.col_idx)


@dataclass
class Report:
    sweeps: int
    stop_reason: int
    levels: int
    beta: float
    delta_fro: list
    products: int
    block_pairs: int
    nnzb_Z: int
    flops: float
    fp64_delta_evals: int = 0
    low_sweeps: int = 0
    launches: int = 0
    gemm_launches: int = 0
    gemm_ms: float = 0.0
    fp64_pairs: int = 0
    tc_launches: int = 0
    tc_ms: float = 0.0
    tc_pairs: int = 0
    resid_fro: float = 0.0
    status: int = 0
    split_launches: int = 0
    split_ms: float = 0.0
    split_pairs: int = 0
    split_slice_pairs: int = 0
    fp64_bytes: float = 0.0
    tc_bytes: float = 0.0
    split_bytes: float = 0.0


def upload(ctx: Context, host) -> DeviceBSR:
    """Copy a host BSR (n, bs, row_ptr, col_idx, val) to the device."""
    rp = np.ascontiguousarray(host.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(host.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(host.val, dtype=np.float64)
    raw = _Bsr()
    ctx.check(ctx.lib.ifac_bsr_upload(ctx.h, int(host.n), int(host.bs), len(rp) - 1, len(ci), rp.ctypes.data,
                                      ci.ctypes.data, v.ctypes.data, ctypes.byref(raw)))
    return DeviceBSR(ctx, raw)


def opts(m: int = 2, max_iter: int = 50, fixed_iters: int = 0, c_rule: int = 0, leaf_size: int = 512,
         prec: int = FP64, profile: bool = False, delta_prec: int | None = None, rinch_rows: int = 0,
         local_delta: bool = False) -> _Opts:
    o = _Opts()
    load().ifac_opts_default(ctypes.byref(o))
    o.m, o.max_iter, o.fixed_iters, o.c_rule, o.leaf_size, o.prec = m, max_iter, fixed_iters, c_rule, leaf_size, prec
    o.profile = int(profile)
    if delta_prec is not None:
        o.delta_prec = delta_prec
    o.rinch_rows = rinch_rows
    o.local_delta = int(local_delta)
    return o


def _report(r: _Report, rc: int) -> Report:
    return Report(r.sweeps, r.stop_reason, r.levels, r.beta, [r.delta_fro[i] for i in range(r.n_delta)],
                  r.products, r.block_pairs, r.nnzb_Z, r.flops, r.fp64_delta_evals, r.low_sweeps, r.launches,
                  r.gemm_launches, r.gemm_ms, r.fp64_pairs, r.tc_launches, r.tc_ms, r.tc_pairs, r.resid_fro, rc,
                  r.split_launches, r.split_ms, r.split_pairs, r.split_slice_pairs, r.fp64_bytes, r.tc_bytes,
                  r.split_bytes)


def bsr_gemm_trunc(ctx: Context, A: DeviceBSR, transA: bool, B: DeviceBSR, transB: bool, alpha: float = 1.0,
                   tau: float = 0.0, prec: int = FP64) -> DeviceBSR:
    C = _Bsr()
    ctx.check(ctx.lib.bsr_gemm_trunc(ctx.h, A.ptr(), int(transA), B.ptr(), int(transB), alpha, tau, prec,
                                     ctypes.byref(C)))
    return DeviceBSR(ctx, C)


def bsr_gemm_sym_trunc(ctx: Context, A: DeviceBSR, transA: bool, B: DeviceBSR, transB: bool, alpha: float = 1.0,
                       tau: float = 0.0, prec: int = FP64) -> DeviceBSR:
    C = _Bsr()
    ctx.check(ctx.lib.bsr_gemm_sym_trunc(ctx.h, A.ptr(), int(transA), B.ptr(), int(transB), alpha, tau, prec,
                                         ctypes.byref(C)))
    return DeviceBSR(ctx, C)


def bsr_add(ctx: Context, alpha: float, A: DeviceBSR, beta: float = 0.0, B: DeviceBSR | None = None,
            gamma: float = 0.0) -> DeviceBSR:
    C = _Bsr()
    ctx.check(ctx.lib.bsr_add(ctx.h, alpha, A.ptr(), beta, B.ptr() if B is not None else None, gamma,
                              ctypes.byref(C)))
    return DeviceBSR(ctx, C)


def bsr_truncate(ctx: Context, A: DeviceBSR, tau: float) -> DeviceBSR:
    C = _Bsr()
    ctx.check(ctx.lib.bsr_truncate(ctx.h, A.ptr(), tau, ctypes.byref(C)))
    return DeviceBSR(ctx, C)


def bsr_fro(ctx: Context, A: DeviceBSR) -> float:
    out = ctypes.c_double()
    ctx.check(ctx.lib.bsr_fro(ctx.h, A.ptr(), ctypes.byref(out)))
    return out.value


def bsr_gershgorin(ctx: Context, A: DeviceBSR) -> float:
    out = ctypes.c_double()
    ctx.check(ctx.lib.bsr_gershgorin(ctx.h, A.ptr(), ctypes.byref(out)))
    return out.value


def leaf_invchol_batched(ctx: Context, S, Z=None, info=None):
    """S: CUDA float64 tensor [count, nl, nl]; returns (Z, info) tensors."""
    import torch
    count, nl = S.shape[0], S.shape[1]
    assert S.is_cuda and S.dtype == torch.float64 and S.is_contiguous()
    if Z is None:
        Z = torch.empty_like(S)
    if info is None:
        info = torch.zeros(count, dtype=torch.int32, device=S.device)
    rc = ctx.lib.leaf_invchol_batched(ctx.h, count, nl, S.data_ptr(), Z.data_ptr(), info.data_ptr())
    if rc != ERR_NOT_SPD:
        ctx.check(rc)
    return Z, info, rc


def inv_factor_refine(ctx: Context, S: DeviceBSR, tau: float, target: float, o: _Opts | None = None):
    Z = _Bsr()
    rep = _Report()
    rc = ctx.check(ctx.lib.inv_factor_refine(ctx.h, S.ptr(), tau, target, ctypes.byref(o or opts()),
                                             ctypes.byref(Z), ctypes.byref(rep)))
    return DeviceBSR(ctx, Z), _report(rep, rc)


def inv_factor_localized(ctx: Context, S: DeviceBSR, tau: float, target: float, o: _Opts | None = None):
    Z = _Bsr()
    rep = _Report()
    rc = ctx.check(ctx.lib.inv_factor_localized(ctx.h, S.ptr(), tau, target, ctypes.byref(o or opts()),
                                                ctypes.byref(Z), ctypes.byref(rep)))
    return DeviceBSR(ctx, Z), _report(rep, rc)


def inv_factor_rinch(ctx: Context, S: DeviceBSR, tau: float, o: _Opts | None = None):
    """Recursive inverse Cholesky (Algorithm 1); opts.leaf_size sets the leaf level."""
    Z = _Bsr()
    rep = _Report()
    rc = ctx.check(ctx.lib.inv_factor_rinch(ctx.h, S.ptr(), tau, ctypes.byref(o or opts()), ctypes.byref(Z),
                                            ctypes.byref(rep)))
    return DeviceBSR(ctx, Z), _report(rep, rc)


def inv_factor_refine_batched(ctx: Context, Ss, tau: float, target: float, o: _Opts | None = None):
    """Refine a list of DeviceBSR together; returns ([Z_k], [Report_k], status)."""
    count = len(Ss)
    ptrs = (ctypes.POINTER(_Bsr) * count)(*[ctypes.pointer(S.raw) for S in Ss])
    Zs = (_Bsr * count)()
    reps = (_Report * count)()
    rc = ctx.check(ctx.lib.inv_factor_refine_batched(ctx.h, count, ctypes.cast(ptrs, ctypes.c_void_p), tau, target,
                                                     ctypes.byref(o or opts()), ctypes.cast(Zs, ctypes.c_void_p),
                                                     ctypes.cast(reps, ctypes.c_void_p)))
    out = []
    for k in range(count):
        z = _Bsr()
        ctypes.pointer(z)[0] = Zs[k]
        out.append(DeviceBSR(ctx, z))
    return out, [_report(reps[k], rc) for k in range(count)], rc


def inv_factor_refine_adjoint(ctx: Context, S, F, K: int = 6, tau: float = 1e-10):
    """(L, Sbar): L = tr(Z_K^T F Z_K) after K frozen-pattern sweeps and
    Sbar = dL/dS on S's pattern (see include/ifac.h).  S, F: DeviceBSR or
    BorrowedBSR."""
    Sb = _Bsr()
    L = ctypes.c_double()
    ctx.check(ctx.lib.inv_factor_refine_adjoint(ctx.h, S.ptr(), F.ptr(), K, tau, ctypes.byref(L), ctypes.byref(Sb)))
    return L.value, DeviceBSR(ctx, Sb)


class BorrowedBSR:
    """An ifac_bsr over caller-owned CUDA tensors (row_ptr, col_idx int32;
    val float64 [nnzb, bs, bs]); the tensors must outlive every call."""

    def __init__(self, n: int, bs: int, row_ptr, col_idx, val):
        self.keep = (row_ptr, col_idx, val)
        self.raw = _Bsr(n, bs, row_ptr.numel() - 1, col_idx.numel(), row_ptr.data_ptr(), col_idx.data_ptr(),
                        val.data_ptr(), None)

    def ptr(self):
        return ctypes.byref(self.raw)


def device_tensors(M: DeviceBSR):
    """Zero-copy torch views (row_ptr, col_idx, val) of a library-owned matrix;
    they keep M alive."""
    import torch

    class _View:
        def __init__(self, ptr, shape, typestr, owner):
            self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}
            self.owner = owner

    nb, nnzb, bs = M.nb, M.nnzb, M.bs
    rp = torch.as_tensor(_View(M.raw.row_ptr, (nb + 1,), "<i4", M), device="cuda")
    ci = torch.as_tensor(_View(M.raw.col_idx or 0, (nnzb,), "<i4", M), device="cuda")
    v = torch.as_tensor(_View(M.raw.val or 0, (nnzb, bs, bs), "<f8", M), device="cuda")
    return rp, ci, v


def inv_factor_resid(ctx: Context, S: DeviceBSR, Z: DeviceBSR) -> float:
    out = ctypes.c_double()
    ctx.check(ctx.lib.inv_factor_resid(ctx.h, S.ptr(), Z.ptr(), ctypes.byref(out)))
    return out.value


def bsr_reblock(ctx: Context, A: DeviceBSR, bs: int) -> DeviceBSR:
    """The same matrix with block size bs (32, 64, 128), exact."""
    out = _Bsr()
    ctx.check(ctx.lib.bsr_reblock(ctx.h, A.ptr(), int(bs), ctypes.byref(out)))
    return DeviceBSR(ctx, out)


def set_schedule(ctx: Context, narrow_kmax: int, narrow_kmax_split: int | None = None) -> None:
    """Tile schedules of bs-64 TF32/BF16 and split products (see
    include/ifac.h); the split schedule defaults to the same value."""
    s = narrow_kmax if narrow_kmax_split is None else narrow_kmax_split
    ctx.check(ctx.lib.ifac_set_schedule(ctx.h, int(narrow_kmax), int(s)))


def autotune_batched(ctx: Context, members, tau: float, o) -> dict:
    """Block size and bs-64 tile schedule of a batched refinement from timed
    probes (sets the schedule on the context); returns the choice and the
    predicted times."""
    arr = (ctypes.POINTER(_Bsr) * len(members))(*[ctypes.pointer(m.raw) for m in members])
    r = _TuneResult()
    ctx.check(ctx.lib.ifac_autotune_batched(ctx.h, len(members), ctypes.cast(arr, ctypes.c_void_p), tau,
                                            ctypes.byref(o), ctypes.byref(r)))
    names = ("default", "super_tiles", "narrow")
    return {"bs": r.bs, "narrow_kmax": r.narrow_kmax, "narrow_kmax_split": r.narrow_kmax_split,
            "probe_ms": {32: r.probe_ms[0], 64: r.probe_ms[1], 128: r.probe_ms[2]},
            "probe64_lp_ms": dict(zip(names, r.probe64_lp_ms)),
            "probe64_split_ms": dict(zip(names, r.probe64_split_ms)),
            "low_sweeps_est": r.low_sweeps_est, "split_evals_est": r.split_evals_est}


def selftest_wait_timeout(ctx: Context, wait_limit: int) -> int:
    """Failure-path self-test of the bounded device waits (include/ifac.h):
    returns the status code (IFAC_ERR_TIMEOUT expected) without raising."""
    return ctx.lib.ifac_selftest_wait_timeout(ctx.h, int(wait_limit))


def leaf_invchol_batched_noalloc(stream: int, S, Z, info) -> int:
    """Allocation-free leaf routine (see include/ifac.h): S, Z float64 CUDA
    tensors [count, nl, nl], info int32 CUDA tensor [count]; enqueues on
    `stream` and returns the status code without waiting."""
    count, nl = S.shape[0], S.shape[1]
    return load().leaf_invchol_batched_noalloc(stream, count, nl, S.data_ptr(), Z.data_ptr(), info.data_ptr())
