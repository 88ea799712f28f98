"""The symmetric block product (bsr_gemm_sym_trunc) through the C ABI: only
the output blocks (I, J) with J >= I are multiplied and block (J, I) is the
transpose of block (I, J); a diagonal block is the product's own (symmetric
up to rounding).  Checked against the CPU oracle's full product.

- Integer operands small enough that every partial sum is exact in FP32 (and
  every operand exact in BF16 and TF32): the result equals the oracle's
  product bit for bit in all four precisions, pattern included.
- Real-valued Z^T (S Z) with S symmetric: within the same element bound as
  the ordinary product, applied to both (I, J) and (J, I), and the blocks off
  the diagonal are exactly symmetric; with truncation every kept block has
  its mirror kept.
"""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
FP64, TF32, BF16, FP64_SPLIT = 0, 1, 2, 3


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac.Context()


def dense(h):
    nb, bs = h.nb, h.bs
    D = np.zeros((nb * bs, nb * bs))
    for I in range(nb):
        for q in range(h.row_ptr[I], h.row_ptr[I + 1]):
            J = h.col_idx[q]
            D[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = h.val[q]
    return D


def _mirror_exact(G, bs):
    """Off the diagonal blocks, G equals its transpose bit for bit."""
    blk = np.arange(G.shape[0]) // bs
    off = blk[:, None] != blk[None, :]
    return np.array_equal(G[off], G.T[off])


def _int_bsr(nb, density, seed, empty_rows=0, n=None):
    h = synth.random_bsr(nb, 64, density, seed=seed, empty_rows=empty_rows, n=n)
    rng = np.random.default_rng(seed + 100)
    return synth.HostBSR(h.n, 64, h.row_ptr, h.col_idx, rng.integers(-3, 4, size=h.val.shape).astype(np.float64))


@pytest.mark.parametrize("prec", [FP64, TF32, BF16, FP64_SPLIT])
def test_sym_exact_integer_gram(ctx, prec):
    """C = A^T A and C = A A^T (ragged n, empty rows): |partial sums| <= 9 K <
    2^24, so every precision is exact and the mirrored blocks equal the
    oracle's own lower blocks."""
    from paper_1901_07993_gb300 import ifac
    nb = 11
    A = _int_bsr(nb, 0.35, seed=5, empty_rows=2, n=nb * 64 - 13)
    dA = ifac.upload(ctx, A)
    for tA, tB in ((True, False), (False, True)):
        ref = oracle.gemm(A, A, tA, tB, -2.0, 0.0)
        got = ifac.bsr_gemm_sym_trunc(ctx, dA, tA, dA, tB, -2.0, 0.0, prec).download()
        assert np.array_equal(got.row_ptr, ref.row_ptr) and np.array_equal(got.col_idx, ref.col_idx)
        assert np.array_equal(got.val, ref.val)


@pytest.mark.parametrize("prec", [FP64, FP64_SPLIT])
def test_sym_congruence_fp64_class(ctx, prec):
    """Z^T (S Z) for a chain overlap S and a random banded Z: FP64-class
    agreement with the oracle's full product in both triangles."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(1500, 64, seed=3)
    Zh = synth.random_bsr(S.nb, 64, 0.3, seed=8, n=S.n)
    X = oracle.gemm(S, Zh, False, False, 1.0, 0.0)
    Xh = synth.HostBSR(X.n, 64, X.row_ptr, X.col_idx, X.val)
    ref = oracle.gemm(Zh, Xh, True, False, 1.0, 0.0)
    got = ifac.bsr_gemm_sym_trunc(ctx, ifac.upload(ctx, Zh), True, ifac.upload(ctx, Xh), False, 1.0, 0.0,
                                  prec).download()
    assert np.array_equal(got.row_ptr, ref.row_ptr) and np.array_equal(got.col_idx, ref.col_idx)
    G, R = dense(got), dense(ref)
    assert _mirror_exact(G, 64)
    # |Z|^T |S| |Z| bounds both the product's rounding and the asymmetry
    # that the rounding of S Z leaves in the oracle's full product
    absZ = np.abs(dense(Zh))
    absb = absZ.T @ (np.abs(dense(S)) @ absZ)
    K = S.nb * 64
    eps = 2.0 ** -53 if prec == FP64 else 2.0 ** -40
    lim = 2 * K * eps * (absb + absb.T) + 1e-300
    assert np.all(np.abs(G - R) <= lim), float((np.abs(G - R) / lim).max())


@pytest.mark.parametrize("prec", [TF32, FP64_SPLIT])
def test_sym_truncation_keeps_mirrors(ctx, prec):
    """delta delta with delta symmetric and tau between block norms: the kept
    pattern is symmetric, every kept block has norm >= tau, and the values
    agree with the oracle's truncated product where both keep the block."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(3000, 64, seed=6)
    St = oracle.truncate(S, 1e-8)
    D = oracle.add(-1.0, St, 0.0, None, 1.0)
    Dh = synth.HostBSR(D.n, 64, D.row_ptr, D.col_idx, D.val)
    full = oracle.gemm(Dh, Dh, False, False, 1.0, 0.0)
    norms = np.sort(np.sqrt((full.val ** 2).sum(axis=(1, 2))))
    tau = float(norms[len(norms) // 3])
    got = ifac.bsr_gemm_sym_trunc(ctx, ifac.upload(ctx, Dh), False, ifac.upload(ctx, Dh), False, 1.0, tau,
                                  prec).download()
    rows = np.repeat(np.arange(got.nb), np.diff(got.row_ptr))
    kept = set(zip(rows.tolist(), got.col_idx.tolist()))
    assert all((j, i) in kept for i, j in kept)
    gn = np.sqrt((got.val ** 2).sum(axis=(1, 2)))
    tol = 1e-3 if prec == TF32 else 1e-12
    assert np.all(gn >= tau * (1 - tol))
    G = dense(got)
    assert _mirror_exact(G, 64)
    R = dense(oracle.truncate(full, tau))
    both = (G != 0) & (R != 0)
    assert np.abs(G - R)[both].max() <= tol * np.abs(R).max()


def test_sym_bs32_unsupported(ctx):
    from paper_1901_07993_gb300 import ifac
    A = synth.random_bsr(4, 32, 0.5, seed=1)
    dA = ifac.upload(ctx, A)
    with pytest.raises(ifac.IfacError) as e:
        ifac.bsr_gemm_sym_trunc(ctx, dA, True, dA, False, 1.0, 0.0, FP64)
    assert e.value.code == ifac.ERR_UNSUPPORTED
