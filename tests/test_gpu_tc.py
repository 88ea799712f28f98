"""Tensor-core (tcgen05) block products with TF32 / BF16 inputs and FP32
accumulation, through the C ABI, against the CPU oracle's FP64 product of the
same inputs rounded the same way (BF16: round-to-nearest-even from FP64;
TF32: FP64 -> FP32 round-to-nearest-even, then round half away from zero to
10 fraction bits).  With identically rounded inputs the only difference left
is FP32 accumulation, bounded element-wise by K * 2^-22 * (|A||B|)_ij, plus
K * 2^-120 for terms below FP32's normal range, which the GPU flushes to zero
(overlap matrices hold entries far below 1e-38)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
TF32, BF16 = 1, 2


def round_bf16(x):
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def round_tf32(x):
    u = x.astype(np.float32).view(np.uint32)
    u = (u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return u.view(np.float32).astype(np.float64)


def rounded(h, prec):
    f = round_tf32 if prec == TF32 else round_bf16
    return synth.HostBSR(h.n, h.bs, h.row_ptr, h.col_idx, f(h.val))


def abs_mat(h):
    return synth.HostBSR(h.n, h.bs, h.row_ptr, h.col_idx, np.abs(h.val))


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac.Context()


def _check(ctx, A, B, tA, tB, prec, alpha=1.0):
    from paper_1901_07993_gb300 import ifac
    ref = oracle.gemm(rounded(A, prec), rounded(B, prec), tA, tB, alpha, 0.0)
    bound = oracle.gemm(abs_mat(rounded(A, prec)), abs_mat(rounded(B, prec)), tA, tB, abs(alpha), 0.0)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), tA, ifac.upload(ctx, B), tB, alpha, 0.0, prec).download()
    assert np.array_equal(got.row_ptr, ref.row_ptr) and np.array_equal(got.col_idx, ref.col_idx)
    kmax = A.nb * A.bs
    err = np.abs(got.val - ref.val)
    lim = kmax * 2.0 ** -22 * bound.val + kmax * 2.0 ** -120
    worst = np.unravel_index(np.argmax(err / lim), err.shape)
    assert np.all(err <= lim), (float(err[worst]), float(lim[worst]), float(ref.val[worst]))
    return np.abs(got.val - oracle.gemm(A, B, tA, tB, alpha, 0.0).val).max()


@pytest.mark.parametrize("prec", [TF32, BF16])
@pytest.mark.parametrize("tA,tB", list(itertools.product([False, True], repeat=2)))
def test_tc_random_blocks(ctx, prec, tA, tB):
    nb = 9
    A = synth.random_bsr(nb, 64, 0.4, seed=31, empty_rows=1, n=nb * 64 - 7)
    B = synth.random_bsr(nb, 64, 0.4, seed=32, empty_rows=2, n=nb * 64 - 7)
    _check(ctx, A, B, tA, tB, prec, alpha=-1.25)


@pytest.mark.parametrize("prec", [TF32, BF16])
def test_tc_overlap_products(ctx, prec):
    """S S and S^T S on a 3D cluster (bs 64): dense-ish tiles, realistic values."""
    S = synth.cluster_overlap(1536, 64, seed=2)
    St = oracle.truncate(S, 1e-10)
    St = synth.HostBSR(St.n, 64, St.row_ptr, St.col_idx, St.val)
    e1 = _check(ctx, St, St, False, False, prec)
    e2 = _check(ctx, St, St, True, False, prec)
    # error against the unrounded FP64 product, stated (not a bound)
    print(f"prec {prec}: max |C - C_fp64| = {max(e1, e2):.3e}")


@pytest.mark.parametrize("prec", [TF32, BF16])
def test_tc_truncation_and_sparse_tiles(ctx, prec):
    """A sparse 1D-chain pattern (most tile blocks missing) with truncation
    (Section 5).  The blocks of S are scaled by powers of two 2^-k, k in
    0..26 (exact, so rounding commutes with the scaling), which spreads the
    product's block norms over about eight decades; tau sits in the widest
    relative gap between the rounded-input oracle product's norms, far wider
    than the FP32-accumulation error, so both precisions keep exactly the
    oracle's blocks."""
    from paper_1901_07993_gb300 import ifac
    rng = np.random.default_rng(40 + prec)
    S0 = synth.chain_overlap(2000, 64, seed=4)
    S = synth.HostBSR(S0.n, 64, S0.row_ptr, S0.col_idx,
                      S0.val * np.ldexp(1.0, -rng.integers(0, 27, size=(S0.nnzb, 1, 1))))
    ref = oracle.gemm(rounded(S, prec), rounded(S, prec), False, False, 1.0, 0.0)
    bound = oracle.gemm(abs_mat(rounded(S, prec)), abs_mat(rounded(S, prec)), False, False, 1.0, 0.0)
    norms = np.sqrt((ref.val ** 2).sum(axis=(1, 2)))
    srt = np.sort(norms)
    sel = srt[(srt > 1e-6 * srt[-1]) & (srt < 1e-1 * srt[-1])]
    k = int(np.argmax(sel[1:] / sel[:-1]))
    tau = float(np.sqrt(sel[k] * sel[k + 1]))
    assert sel[k + 1] > 1.05 * sel[k], "the scaling must open a gap between block norms"
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, S), False, ifac.upload(ctx, S), False, 1.0, tau, prec).download()
    keep = oracle.truncate(ref, tau)
    assert 0 < keep.nnzb < ref.nnzb
    assert np.array_equal(got.col_idx, keep.col_idx) and np.array_equal(got.row_ptr, keep.row_ptr)
    mask = ~(norms < tau)
    lim = S.nb * 64 * 2.0 ** -22 * bound.val[mask] + S.nb * 64 * 2.0 ** -120
    assert np.all(np.abs(got.val - ref.val[mask]) <= lim)


@pytest.mark.parametrize("prec", [TF32, BF16])
def test_tc_input_rounding_exact(ctx, prec):
    """C = A I on the tensor cores is A rounded to the input format, exactly:
    ties at the rounding position (to even for BF16, the FP32 step of TF32;
    away from zero for TF32's last step), carries into the exponent, signed
    values and magnitudes near and below 2^-126 (zero below)."""
    from paper_1901_07993_gb300 import ifac
    rng = np.random.default_rng(7)
    nb, bs = 2, 64
    v = rng.standard_normal((nb * nb, bs, bs))
    special = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -24,
                        1 + 3 * 2.0 ** -24, 2 - 2.0 ** -9, 2 - 2.0 ** -12, 2.0 ** -126, 1.5 * 2.0 ** -126,
                        2.0 ** -127, 0.0, -0.0, 3.0e38, 1e-300, 2.0 ** 100 * (1 + 2.0 ** -8)])
    flat = v.reshape(-1)
    flat[:len(special)] = special
    flat[len(special):2 * len(special)] = -special
    rp = np.arange(0, nb * nb + 1, nb, dtype=np.int32)
    ci = np.tile(np.arange(nb, dtype=np.int32), nb)
    A = synth.HostBSR(nb * bs, bs, rp, ci, v)
    eye = np.zeros((nb, bs, bs))
    eye[:] = np.eye(bs)
    I = synth.HostBSR(nb * bs, bs, np.arange(nb + 1, dtype=np.int32), np.arange(nb, dtype=np.int32), eye)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), False, ifac.upload(ctx, I), False, 1.0, 0.0, prec).download()
    want = rounded(A, prec).val
    want = np.where(np.abs(want) < 2.0 ** -126, 0.0, want)
    assert np.array_equal(got.val, want)


@pytest.mark.parametrize("prec", [TF32, BF16, 3])
def test_tc_large_pattern_csr_lookups(ctx, prec):
    """nb = 2188 block rows (nb^2 above the dense-map limit of 4M): the tile
    plan finds blocks by binary search in the CSR patterns.  TF32/BF16 against
    the rounded-input bound, the split product against the FP64 product."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(140000, 64, seed=9)
    S = oracle.truncate(S, 1e-12)
    S = synth.HostBSR(S.n, 64, S.row_ptr, S.col_idx, S.val)
    dS = ifac.upload(ctx, S)
    got = ifac.bsr_gemm_trunc(ctx, dS, True, dS, False, 1.0, 0.0, prec).download()
    if prec == 3:
        ref = oracle.gemm(S, S, True, False, 1.0, 0.0)
        assert np.array_equal(got.col_idx, ref.col_idx) and np.array_equal(got.row_ptr, ref.row_ptr)
        assert np.abs(got.val - ref.val).max() <= 1e-13 * np.abs(ref.val).max()
    else:
        _check(ctx, S, S, True, False, prec)


@pytest.mark.parametrize("bs", [32, 128])
@pytest.mark.parametrize("prec", [TF32, BF16])
@pytest.mark.parametrize("tA,tB", [(False, False), (True, False), (False, True)])
def test_tc_block_sizes_32_and_128(ctx, bs, prec, tA, tB):
    """The narrow-tile kernel at bs 32 (tiles of 4 x 2 blocks; BF16 rows of
    64 bytes, 64-byte swizzle) and bs 128 (tiles of one block, K in two
    chunks): random patterns with empty rows, a ragged last tile (nb not a
    multiple of the tile's block rows) and n not a multiple of bs."""
    nb = 11 if bs == 32 else 5
    A = synth.random_bsr(nb, bs, 0.45, seed=60 + bs, empty_rows=1, n=nb * bs - 5)
    B = synth.random_bsr(nb, bs, 0.45, seed=61 + bs, empty_rows=1, n=nb * bs - 5)
    _check(ctx, A, B, tA, tB, prec, alpha=0.75)


@pytest.mark.parametrize("bs", [32, 128])
@pytest.mark.parametrize("prec", [TF32, BF16])
def test_tc_block_sizes_overlap_and_rounding(ctx, bs, prec):
    """S S on a 1D chain and a dense 3D cluster at bs 32 / 128 against the
    rounded-input bound, and C = A I reproducing the rounded A exactly."""
    from paper_1901_07993_gb300 import ifac
    for S in (synth.chain_overlap(3000, bs, seed=5), synth.cluster_overlap(1024, bs, seed=6)):
        St = oracle.truncate(S, 1e-10)
        St = synth.HostBSR(St.n, bs, St.row_ptr, St.col_idx, St.val)
        _check(ctx, St, St, False, False, prec)
    rng = np.random.default_rng(bs + prec)
    nb = 3
    v = rng.standard_normal((nb * nb, bs, bs))
    rp = np.arange(0, nb * nb + 1, nb, dtype=np.int32)
    ci = np.tile(np.arange(nb, dtype=np.int32), nb)
    A = synth.HostBSR(nb * bs, bs, rp, ci, v)
    eye = np.zeros((nb, bs, bs))
    eye[:] = np.eye(bs)
    I = synth.HostBSR(nb * bs, bs, np.arange(nb + 1, dtype=np.int32), np.arange(nb, dtype=np.int32), eye)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), False, ifac.upload(ctx, I), False, 1.0, 0.0, prec).download()
    assert np.array_equal(got.val, rounded(A, prec).val)


@pytest.mark.parametrize("schedule", [0, 1 << 30])
@pytest.mark.parametrize("prec", [TF32, BF16])
def test_tc_schedules_bs64(ctx, schedule, prec):
    """bs 64 TF32/BF16 products under the super-tile-only and narrow-only
    schedules, dense and banded patterns, against the rounded-input bound."""
    from paper_1901_07993_gb300 import ifac
    ifac.set_schedule(ctx, schedule)
    try:
        A = synth.random_bsr(24, 64, 1.0, seed=77)
        B = synth.random_bsr(24, 64, 0.3, seed=78)
        _check(ctx, A, B, False, True, prec)
        S = synth.chain_overlap(2000, 64, seed=4)
        _check(ctx, S, S, True, False, prec)
    finally:
        ifac.set_schedule(ctx, -1)
