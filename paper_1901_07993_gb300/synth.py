"""Seeded synthetic inputs: Gaussian-overlap matrices in block-sparse form.

This module generates the input matrix S for the factorization path and for
its CPU oracle.  It holds none of the method's arithmetic: no products, no
refinement, and no truncation at the method's threshold tau (S is returned
with a generation cutoff ``drop`` far below tau; applying tau is step one of
the method itself, Section 5 of the paper: S is truncated with the same
threshold as the products, then factorized).

The paper's matrices (STO-3G overlap of Glu-Ala helices and water clusters,
Section 5) are not available; these stand in for them:

* ``chain``: a quasi-linear 1D chain of centres, spacing 1.4 bohr with
  uniform +-0.1 jitter (the helices);
* ``cluster``: a 3D cluster drawn by random sequential addition in a cube at
  0.1 points per bohr^3 with minimum separation 1.8 bohr, ordered by recursive
  coordinate bisection (the water clusters).

Exponents cycle through (0.17, 0.62, 3.4) by generation index.  The overlap
of two normalized s-type Gaussians is
``(2 sqrt(a b)/(a+b))^1.5 * exp(-a b/(a+b) r^2)``, so S_ii = 1 and S is SPD.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None

EXPONENTS = (0.17, 0.62, 3.4)
CHAIN_SPACING = 1.4
CHAIN_JITTER = 0.1
CLUSTER_DENSITY = 0.1
CLUSTER_DMIN = 1.8
GEN_DROP = 1e-14


def build(force: bool = False) -> str:
    """Compile synth.c into _synth.so next to it (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, dbl, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.synth_rng_draw.argtypes = [u64, i64]
        lib.synth_rng_draw.restype = u64
        lib.synth_chain.argtypes = [i64, dbl, dbl, u64, p]
        lib.synth_chain.restype = None
        lib.synth_rsa_cube.argtypes = [i64, dbl, dbl, u64, i64, p]
        lib.synth_rsa_cube.restype = i64
        lib.synth_rcb_order.argtypes = [i64, p, ctypes.c_int, p]
        lib.synth_rcb_order.restype = None
        lib.synth_overlap_bsr.argtypes = [i64, p, p, ctypes.c_int, dbl]
        lib.synth_overlap_bsr.restype = p
        lib.synth_bsr_nnzb.argtypes = [p]
        lib.synth_bsr_nnzb.restype = i64
        lib.synth_bsr_take.argtypes = [p, ctypes.c_int, p, p, p]
        lib.synth_bsr_take.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


@dataclass
class HostBSR:
    """A square block-sparse matrix in host memory.

    n: logical dimension; bs: block size; nb = ceil(n/bs) block rows/cols.
    row_ptr[nb+1] (int32), col_idx[nnzb] (int32, sorted within a row),
    val[nnzb, bs, bs] (float64, each block row-major).  Rows/cols past n
    (padding of the last block) carry a unit diagonal.
    """
    n: int
    bs: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nb(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnzb(self) -> int:
        return len(self.col_idx)

    def to_dense(self) -> np.ndarray:
        nb, bs = self.nb, self.bs
        d = np.zeros((nb * bs, nb * bs))
        for i in range(nb):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                j = self.col_idx[p]
                d[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = self.val[p]
        return d


@dataclass
class Geometry:
    xyz: np.ndarray    # [n, 3] bohr, in matrix order
    alpha: np.ndarray  # [n] Gaussian exponents, in matrix order


def rng_draw(seed: int, k: int) -> int:
    """k-th raw 64-bit SplitMix64 draw of stream ``seed`` (k >= 1)."""
    return int(_load().synth_rng_draw(seed, k))


def exponents(n: int) -> np.ndarray:
    return np.array([EXPONENTS[i % 3] for i in range(n)], dtype=np.float64)


def chain(n: int, seed: int = 0) -> Geometry:
    xyz = np.zeros((n, 3))
    _load().synth_chain(n, CHAIN_SPACING, CHAIN_JITTER, seed, _ptr(xyz))
    return Geometry(xyz, exponents(n))


def cluster(n: int, bs: int, seed: int = 0) -> Geometry:
    """3D random-sequential-addition cluster in RCB order for block size bs."""
    xyz = np.zeros((n, 3))
    placed = _load().synth_rsa_cube(n, CLUSTER_DENSITY, CLUSTER_DMIN, seed, 2000 * n + 10**6, _ptr(xyz))
    if placed != n:
        raise RuntimeError(f"random sequential addition placed {placed} of {n} points")
    perm = np.zeros(n, dtype=np.int64)
    _load().synth_rcb_order(n, _ptr(xyz), bs, _ptr(perm))
    alpha = exponents(n)  # by generation index, before reordering
    return Geometry(np.ascontiguousarray(xyz[perm]), np.ascontiguousarray(alpha[perm]))


def overlap_bsr(geom: Geometry, bs: int, drop: float = GEN_DROP) -> HostBSR:
    n = geom.xyz.shape[0]
    xyz = np.ascontiguousarray(geom.xyz, dtype=np.float64)
    alpha = np.ascontiguousarray(geom.alpha, dtype=np.float64)
    lib = _load()
    h = lib.synth_overlap_bsr(n, _ptr(xyz), _ptr(alpha), bs, drop)
    if not h:
        raise MemoryError("synth_overlap_bsr failed")
    nb = (n + bs - 1) // bs
    nnzb = lib.synth_bsr_nnzb(h)
    row_ptr = np.zeros(nb + 1, dtype=np.int32)
    col_idx = np.zeros(nnzb, dtype=np.int32)
    val = np.zeros((nnzb, bs, bs), dtype=np.float64)
    lib.synth_bsr_take(h, bs, _ptr(row_ptr), _ptr(col_idx), _ptr(val))
    return HostBSR(n, bs, row_ptr, col_idx, val)


def chain_overlap(n: int, bs: int, seed: int = 0) -> HostBSR:
    return overlap_bsr(chain(n, seed), bs)


def cluster_overlap(n: int, bs: int, seed: int = 0) -> HostBSR:
    return overlap_bsr(cluster(n, bs, seed), bs)


def random_bsr(nb: int, bs: int, density: float, seed: int, n: int | None = None,
               empty_rows: int = 0, scale: float = 1.0) -> HostBSR:
    """Random block-sparse test matrix (for product tests): each block present
    with probability ``density``; ``empty_rows`` block rows are left empty;
    values N(0,1)*scale.  Uses numpy's PCG64 seeded generator."""
    rng = np.random.default_rng(seed)
    mask = rng.random((nb, nb)) < density
    if empty_rows:
        rows = rng.choice(nb, size=min(empty_rows, nb), replace=False)
        mask[rows, :] = False
    row_ptr = np.zeros(nb + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(mask.sum(axis=1))
    col_idx = np.nonzero(mask)[1].astype(np.int32)
    val = rng.standard_normal((len(col_idx), bs, bs)) * scale
    return HostBSR(n if n is not None else nb * bs, bs, row_ptr, col_idx, val)


def fock_like(S: HostBSR, seed: int = 5) -> HostBSR:
    """Symmetric matrix on the block pattern of S with entries N(0,1) * S_ij
    (a stand-in for a Fock-like matrix).  Blocks (I, J), I <= J, draw their
    N(0,1) factors in CSR order from numpy's PCG64 with the given seed;
    diagonal blocks are symmetrized and block (J, I) is the transpose."""
    rng = np.random.default_rng(seed)
    nb, bs = S.nb, S.bs
    rows = np.repeat(np.arange(nb), np.diff(S.row_ptr))
    pos = {(int(i), int(j)): p for p, (i, j) in enumerate(zip(rows, S.col_idx))}
    val = np.zeros_like(S.val)
    for p, (i, j) in enumerate(zip(rows, S.col_idx)):
        if i > j:
            continue
        g = rng.standard_normal((bs, bs))
        if i == j:
            g = np.triu(g) + np.triu(g, 1).T
        val[p] = g * S.val[p]
        if i != j:
            q = pos.get((int(j), int(i)))
            if q is None:
                raise ValueError("S pattern is not symmetric")
            val[q] = val[p].T
    return HostBSR(S.n, S.bs, S.row_ptr.copy(), S.col_idx.copy(), val)
