"""FP64-accurate block products on the tensor cores (error-free splitting into
BF16 slices, Ozaki et al. 2012) through the C ABI, against the CPU oracle's
FP64 product.

Bound used element-wise: every scalar row i of op(A) is split relative to a
power of two sigma_i < 2 max_k |a_ik|, every column j of op(B) relative to
tau_j < 2 max_k |b_kj|; the dropped slice pairs and the split remainders cost
at most about 2^-(7 NS - 3) sigma_i tau_j per product term (NS slices; 2^-46
for the default 7), and the conversion of the fixed-point sum rounds once per
unit and window (at most 16 ceil(K/16) times).  With a factor 4 of margin:
    |C - C_ref| <= K 2^-(7 NS - 5) r_i c_j + (16 ceil(K/16) + K) 2^-53 (|A||B|)_ij
with r_i = max_k |a_ik|, c_j = max_k |b_kj|, K = scalar inner length."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
FP64_SPLIT = 3


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


def _check(ctx, A, B, tA, tB, alpha=1.0, ns=7):
    from paper_1901_07993_gb300 import ifac
    ref = oracle.gemm(A, B, tA, tB, alpha, 0.0)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), tA, ifac.upload(ctx, B), tB, alpha, 0.0,
                              FP64_SPLIT).download()
    assert np.array_equal(got.row_ptr, ref.row_ptr) and np.array_equal(got.col_idx, ref.col_idx)
    Ad, Bd = dense(A), dense(B)
    Ad = Ad.T if tA else Ad
    Bd = Bd.T if tB else Bd
    r = np.abs(Ad).max(axis=1)
    c = np.abs(Bd).max(axis=0)
    absab = np.abs(Ad) @ np.abs(Bd)
    K = A.nb * A.bs
    lim_d = abs(alpha) * (K * 2.0 ** -(7 * ns - 5) * np.outer(r, c) + (16 * -(-A.nb // 16) + K) * 2.0 ** -53 * absab)
    bs = A.bs
    worst = 0.0
    for I in range(A.nb):
        for q in range(ref.row_ptr[I], ref.row_ptr[I + 1]):
            J = ref.col_idx[q]
            lim = lim_d[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs]
            err = np.abs(got.val[q] - ref.val[q])
            assert np.all(err <= lim), (I, J, float(err.max()), float(lim.min()))
            worst = max(worst, float((err / np.maximum(lim, 1e-300)).max()))
    return worst, np.abs(got.val - ref.val).max() / max(np.abs(ref.val).max(), 1e-300)


@pytest.mark.parametrize("tA,tB", list(itertools.product([False, True], repeat=2)))
def test_split_random_blocks(ctx, tA, tB):
    """Ragged n, empty rows, all four transpose cases, alpha not a power of two."""
    nb = 9
    A = synth.random_bsr(nb, 64, 0.4, seed=41, empty_rows=1, n=nb * 64 - 7)
    B = synth.random_bsr(nb, 64, 0.4, seed=42, empty_rows=2, n=nb * 64 - 7)
    _, rel = _check(ctx, A, B, tA, tB, alpha=-1.25)
    assert rel < 1e-13  # FP64 class (TF32 and BF16 products give 1e-4 .. 1e-2)


@pytest.mark.parametrize("ns", [3, 4, 5, 8])
def test_split_slice_count(ctx, ns):
    """Fewer or more slices move the bound by 2^-7 per slice; 8 slices use
    36 pairs in 16 accumulation units, 3 slices 6 pairs in 4 units."""
    A = synth.random_bsr(20, 64, 0.5, seed=51)
    B = synth.random_bsr(20, 64, 0.5, seed=52)
    ctx.set_split_slices(ns)
    try:
        _, rel = _check(ctx, A, B, False, True, alpha=0.75, ns=ns)
    finally:
        ctx.set_split_slices(7)
    assert rel < {3: 1e-4, 4: 1e-6, 5: 1e-9, 8: 1e-13}[ns]


def test_split_truncation(ctx):
    """Norm-based truncation after the split product keeps the oracle's blocks
    (block magnitudes spread over 10^-8 .. 1, threshold in a gap between
    product norms far above the product's absolute error)."""
    from paper_1901_07993_gb300 import ifac
    rng = np.random.default_rng(48)

    def spread(h):
        v = h.val * 10.0 ** -rng.uniform(0, 8, size=(h.nnzb, 1, 1))
        return synth.HostBSR(h.n, h.bs, h.row_ptr, h.col_idx, v)

    A = spread(synth.random_bsr(12, 64, 0.35, seed=49))
    B = spread(synth.random_bsr(12, 64, 0.35, seed=50))
    ref = oracle.gemm(A, B, False, False, 1.0, 0.0)
    norms = np.sort(np.sqrt((ref.val ** 2).sum(axis=(1, 2))))
    sel = norms[(norms > 1e-6 * norms[-1]) & (norms < 1e-1 * norms[-1])]
    k = int(np.argmax(sel[1:] / sel[:-1]))
    tau = np.sqrt(sel[k] * sel[k + 1])
    assert sel[k + 1] > 1.01 * sel[k]
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), False, ifac.upload(ctx, B), False, 1.0, tau,
                              FP64_SPLIT).download()
    keep = oracle.truncate(ref, tau)
    assert 0 < keep.nnzb < ref.nnzb
    assert np.array_equal(got.col_idx, keep.col_idx) and np.array_equal(got.row_ptr, keep.row_ptr)
    assert np.abs(got.val - keep.val).max() <= 1e-13 * np.abs(keep.val).max()


def test_split_many_k_windows(ctx):
    """A dense 40 x 40 block product: 40 K steps per tile, three windows of 16."""
    A = synth.random_bsr(40, 64, 1.0, seed=43)
    B = synth.random_bsr(40, 64, 1.0, seed=44)
    _, rel = _check(ctx, A, B, False, True)
    assert rel < 1e-13  # FP64 class (TF32 and BF16 products give 1e-4 .. 1e-2)


def test_split_wide_dynamic_range(ctx):
    """Rows and columns scaled over 2^-300 .. 2^300: the per-row/column
    power-of-two scales keep every slice product exact."""
    rng = np.random.default_rng(45)
    A = synth.random_bsr(6, 64, 0.6, seed=46)
    B = synth.random_bsr(6, 64, 0.6, seed=47)
    rs = np.ldexp(1.0, rng.integers(-300, 300, size=6 * 64))
    cs = np.ldexp(1.0, rng.integers(-300, 300, size=6 * 64))
    Av = A.val.copy()
    for I in range(A.nb):
        for q in range(A.row_ptr[I], A.row_ptr[I + 1]):
            Av[q] *= rs[I * 64:(I + 1) * 64, None]
    Bv = B.val.copy()
    for I in range(B.nb):
        for q in range(B.row_ptr[I], B.row_ptr[I + 1]):
            J = B.col_idx[q]
            Bv[q] *= cs[None, J * 64:(J + 1) * 64]
    A = synth.HostBSR(A.n, 64, A.row_ptr, A.col_idx, Av)
    B = synth.HostBSR(B.n, 64, B.row_ptr, B.col_idx, Bv)
    _check(ctx, A, B, False, False)


def test_split_overlap_delta(ctx):
    """delta = I - Z^T S Z from a converged FP64 refinement: the products
    carry the FP64 accuracy that the low-precision formats lose."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(1500, 64, seed=4)
    Sd = ifac.upload(ctx, S)
    Z, _ = ifac.inv_factor_refine(ctx, Sd, 1e-12, 1e-12, ifac.opts())
    Zh = Z.download()
    X = oracle.gemm(S, Zh, False, False, 1.0, 0.0)
    _check(ctx, S, Zh, False, False)
    worst, rel = _check(ctx, Zh, X, True, False)
    assert rel < 1e-13  # FP64 class (TF32 and BF16 products give 1e-4 .. 1e-2)


@pytest.mark.parametrize("nb", [16, 17])
def test_split_exact_at_fp32_bound(ctx, nb):
    """All entries 1 - 2^-9: the leading slices are 128 and -32, so the first
    unit's accumulator reaches exactly 2^24 over a full window of 16 K blocks
    (1024 terms); the product K (1 - 2^-9)^2 is representable and must come
    out exact (nb = 17 adds a one-block second window).  The sums (about
    1000 sigma tau) overflow the first, finer fixed-point scale, so this also
    runs the redo with the safe scale."""
    from paper_1901_07993_gb300 import ifac
    n = nb * 64
    v = 1.0 - 2.0 ** -9
    rp = np.arange(0, nb * nb + 1, nb, dtype=np.int32)
    ci = np.tile(np.arange(nb, dtype=np.int32), nb)
    A = synth.HostBSR(n, 64, rp, ci, np.full((nb * nb, 64, 64), v))
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, A), False, ifac.upload(ctx, A), True, 1.0, 0.0,
                              FP64_SPLIT).download()
    assert np.all(got.val == n * v * v)


def _rel(gpu_host, ref) -> float:
    a = oracle.Mat(gpu_host.n, gpu_host.bs, gpu_host.row_ptr, gpu_host.col_idx, gpu_host.val).to_dense()
    b = ref.to_dense()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_split_refine_matches_oracle(ctx):
    """The FP64 refinement with every product on the split kernel keeps the
    FP64 parity bar: same sweeps, delta norms, ||Z - Z_oracle||_F <= 1e-10 ||Z||_F."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(2048, 64, seed=0)
    Z_ref, rep_ref = oracle.irsi(S, m=2, tau=1e-12, target=1e-10)
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), 1e-12, 1e-10, ifac.opts(prec=FP64_SPLIT))
    assert rep.sweeps == rep_ref.sweeps and rep.stop_reason == rep_ref.stop_reason
    # the split products' error is relative to row and column maxima, not to
    # (|A||B|)_ij, so for these decaying factors the delta floor is about
    # 2e-12 here (FP64 pipe: 3e-13); the norms agree down to that floor
    assert np.allclose(rep.delta_fro, rep_ref.delta_fro, rtol=1e-6, atol=1e-11)
    assert _rel(Z.download(), Z_ref) <= 1e-10
    assert rep.split_pairs == rep.block_pairs and rep.fp64_pairs == 0 and rep.tc_pairs == 0
    assert rep.split_slice_pairs == 28 * rep.split_pairs  # every product with 7 slices


def test_split_localized_matches_oracle(ctx):
    from paper_1901_07993_gb300 import ifac
    S = synth.cluster_overlap(768, 64, seed=0)
    Z_ref, rep_ref = oracle.lif(S, tau=1e-8, target=1e-10, leaf_size=128)
    Z, rep = ifac.inv_factor_localized(ctx, ifac.upload(ctx, S), 1e-8, 1e-10,
                                       ifac.opts(leaf_size=128, prec=FP64_SPLIT))
    assert rep.levels == rep_ref.levels and rep.sweeps == rep_ref.sweeps
    assert _rel(Z.download(), Z_ref) <= 1e-10


@pytest.mark.parametrize("n", [8192, 65536])
def test_split_delta_phase_of_mixed_schedule(ctx, n):
    """TF32 sweeps with the FP64-phase delta on the split kernel meet the
    1e-10 target like the FP64 pipe does (the direct residual, FP64 products)."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, 64, seed=1)
    dS = ifac.upload(ctx, S)
    res = {}
    for dp in (0, FP64_SPLIT):
        Z, rep = ifac.inv_factor_refine(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=1, delta_prec=dp))
        assert rep.fp64_delta_evals >= 1 and rep.stop_reason == ifac.STOP_TARGET
        if dp:  # early evaluations may take fewer than 7 slices, never more
            assert 6 * rep.split_pairs <= rep.split_slice_pairs <= 28 * rep.split_pairs
            print(f"n {n}: slice pairs per block pair {rep.split_slice_pairs / rep.split_pairs:.2f}")
        res[dp] = ifac.inv_factor_resid(ctx, dS, Z)
        assert res[dp] <= 1e-10
    print(f"n {n}: resid fp64-pipe delta {res[0]:.3e}, split delta {res[FP64_SPLIT]:.3e}")


@pytest.mark.parametrize("bs", [32, 128])
@pytest.mark.parametrize("tA,tB", [(False, False), (True, False), (False, True), (True, True)])
def test_split_block_sizes_32_and_128(ctx, bs, tA, tB):
    """The narrow split kernel at bs 32 (tiles of 4 x 2 blocks, 64-byte rows)
    and bs 128 (one block row by half a block column, the two halves in one
    CTA, K in two chunks): ragged n, empty rows, alpha not a power of two."""
    nb = 11 if bs == 32 else 5
    A = synth.random_bsr(nb, bs, 0.4, seed=71 + bs, empty_rows=1, n=nb * bs - 7)
    B = synth.random_bsr(nb, bs, 0.4, seed=72 + bs, empty_rows=2, n=nb * bs - 7)
    _, rel = _check(ctx, A, B, tA, tB, alpha=-1.25)
    assert rel < 1e-13


@pytest.mark.parametrize("bs,nb", [(32, 40), (128, 12)])
def test_split_many_windows_block_sizes(ctx, bs, nb):
    """Dense products whose tiles span several exact windows (at most 1024 K
    elements and 8 accumulation units per window: 14 blocks of 32, 3 of 128):
    the epilogue carries the 64-bit sums from window to window."""
    A = synth.random_bsr(nb, bs, 1.0, seed=73)
    B = synth.random_bsr(nb, bs, 1.0, seed=74)
    _, rel = _check(ctx, A, B, False, True)
    assert rel < 1e-13


@pytest.mark.parametrize("bs", [32, 128])
def test_split_refine_block_sizes_match_oracle(ctx, bs):
    """IRSI with every product on the split kernel (prec = IFAC_FP64_SPLIT)
    at bs 32 and 128: the FP64 oracle's factor within 1e-10, same sweeps."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(2048, bs, seed=3)
    tau, target = 1e-12, 1e-10
    Z_ref, rep_ref = oracle.irsi(S, tau=tau, target=target)
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), tau, target, ifac.opts(prec=FP64_SPLIT))
    assert rep.sweeps == rep_ref.sweeps and rep.split_launches > 0
    a = Z.download()
    za = oracle.Mat(a.n, bs, a.row_ptr, a.col_idx, a.val).to_dense()
    zr = Z_ref.to_dense()
    assert np.linalg.norm(za - zr) / np.linalg.norm(zr) <= 1e-10


@pytest.mark.parametrize("schedule", [-1, 0, 1 << 30])
def test_split_schedules_bs64(ctx, schedule):
    """bs 64 under each tile schedule: default (narrow tiles for every split
    product), super-tiles only (windowed, fixed-point sums in HBM), and narrow
    tiles up to an explicit K length (the narrow kernel runs the dense
    product window by window)."""
    from paper_1901_07993_gb300 import ifac
    A = synth.random_bsr(30, 64, 1.0, seed=75)
    B = synth.random_bsr(30, 64, 1.0, seed=76)
    ifac.set_schedule(ctx, schedule)
    try:
        _, rel = _check(ctx, A, B, False, True)
        _, rel2 = _check(ctx, A, B, True, False, alpha=0.3)
    finally:
        ifac.set_schedule(ctx, -1)
    assert rel < 1e-13 and rel2 < 1e-13


@pytest.mark.parametrize("schedule", [-1, 0])
def test_split_delta_of_dense_cluster_factor(ctx, schedule):
    """||I - Z^T S Z||_F of a dense 3D-cluster factor (n = 3072, bs 64, about
    2300 blocks per product) from split products, under the default schedule
    (narrow tiles, 8 exact windows per tile) and super-tiles only, against the same residual from FP64-pipe products.  With 8 slices
    they agree to 1e-11; with 7 (2^-7 less) to 1e-9 -- on dense operands the
    split error of the delta norm is about 270 x the chain-derived estimate,
    which is why a refinement confirms a stop at the target with all slices
    and dense workloads use 8.  Both schedules give the same residual."""
    from paper_1901_07993_gb300 import ifac
    S = synth.cluster_overlap(3072, 64, seed=12)
    dS = ifac.upload(ctx, S)
    Z, _ = ifac.inv_factor_refine(ctx, dS, 1e-14, 1e-11, ifac.opts(max_iter=80))
    r64 = ifac.inv_factor_resid(ctx, dS, Z)
    ifac.set_schedule(ctx, schedule)
    try:
        for ns, tol in ((7, 1e-9), (8, 1e-11)):
            ctx.set_split_slices(ns)
            X = ifac.bsr_gemm_trunc(ctx, dS, False, Z, False, 1.0, 0.0, FP64_SPLIT)
            Y = ifac.bsr_gemm_trunc(ctx, Z, True, X, False, 1.0, 0.0, FP64_SPLIT)
            D = ifac.bsr_add(ctx, -1.0, Y, 0.0, None, 1.0)
            rs = ifac.bsr_fro(ctx, D)
            print(f"schedule {schedule} ns {ns}: split {rs:.3e} fp64 {r64:.3e}")
            assert abs(rs - r64) <= tol, (ns, rs, r64)
    finally:
        ifac.set_schedule(ctx, -1)
        ctx.set_split_slices(7)
