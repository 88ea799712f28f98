"""Re-blocking (bsr_reblock) and the batched autotuner through the C ABI.

bsr_reblock must return the same matrix: the dense padded matrices are equal
element by element (padding rows the new block size adds carry a unit
diagonal), no stored block is all zero unless diagonal, and going there and
back returns the original blocks exactly.  The autotuner must return one of
the three block sizes with positive probe times and leave its schedule on the
context; the batch refined at that block size reaches the target."""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac.Context()


def dense_padded(h):
    nb, bs = h.nb, h.bs
    D = np.zeros((nb * bs, nb * bs))
    for I in range(nb):
        for q in range(h.row_ptr[I], h.row_ptr[I + 1]):
            J = h.col_idx[q]
            D[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = h.val[q]
    return D


@pytest.mark.parametrize("bs_in,bs_out,n", [(64, 32, 1000), (64, 128, 1000), (32, 128, 1100), (128, 32, 1100),
                                            (32, 64, 4096), (128, 64, 777)])
def test_reblock_is_exact(ctx, bs_in, bs_out, n):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs_in, seed=8)
    R = ifac.bsr_reblock(ctx, ifac.upload(ctx, S), bs_out).download()
    assert R.bs == bs_out and len(R.row_ptr) - 1 == -(-n // bs_out)
    Din, Dout = dense_padded(S), dense_padded(R)
    m = min(Din.shape[0], Dout.shape[0])
    assert np.array_equal(Din[:m, :m], Dout[:m, :m])
    # padding rows the output adds past the input's padded size: unit diagonal only
    if Dout.shape[0] > m:
        tail = Dout[m:, :]
        assert np.array_equal(tail[:, m:], np.eye(Dout.shape[0] - m)) and not tail[:, :m].any()
    rows = np.repeat(np.arange(len(R.row_ptr) - 1), np.diff(R.row_ptr))
    nonzero = np.any(R.val != 0, axis=(1, 2))  # (entries near 1e-160 occur: their squares underflow)
    assert np.all(nonzero | (rows == R.col_idx))
    # there and back gives the original blocks
    if Dout.shape[0] == Din.shape[0]:
        B = ifac.bsr_reblock(ctx, ifac.upload(ctx, R), bs_in).download()
        assert np.array_equal(dense_padded(B), Din)


def test_reblock_3d_cluster_products_agree(ctx):
    """The product of re-blocked operands is the re-blocked product (FP64,
    no truncation): checks the patterns' consistency on a 3D cluster."""
    from paper_1901_07993_gb300 import ifac
    S = synth.cluster_overlap(1024, 64, seed=9)
    dS = ifac.upload(ctx, S)
    C64 = ifac.bsr_gemm_trunc(ctx, dS, False, dS, False, 1.0, 0.0, 0)
    S32 = ifac.bsr_reblock(ctx, dS, 32)
    C32 = ifac.bsr_gemm_trunc(ctx, S32, False, S32, False, 1.0, 0.0, 0)
    a, b = dense_padded(C64.download()), dense_padded(C32.download())
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_autotune_and_batch_at_the_chosen_block_size(ctx):
    from paper_1901_07993_gb300 import ifac
    members = []
    for j, n in enumerate((700, 1500, 2600, 900, 2100, 1200)):
        members.append(synth.chain_overlap(n, 64, seed=30 + j) if j % 2 == 0 else
                       synth.cluster_overlap(n, 64, seed=30 + j))
    dS = [ifac.upload(ctx, S) for S in members]
    o = ifac.opts(prec=1, max_iter=100)
    tune = ifac.autotune_batched(ctx, dS, 1e-12, o)
    print("autotune:", tune)
    assert tune["bs"] in (32, 64, 128)
    assert all(v > 0 for v in tune["probe_ms"].values())
    assert all(v > 0 for v in tune["probe64_lp_ms"].values())
    assert all(v > 0 for v in tune["probe64_split_ms"].values())
    bs = tune["bs"]
    dT = [S if bs == 64 else ifac.bsr_reblock(ctx, S, bs) for S in dS]
    Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dT, 1e-12, 1e-10, o)
    assert rc in (ifac.OK, ifac.WARN_TARGET_NOT_MET)
    for S, Z in zip(members, Zs):
        # the oracle's FP64 residual, with S blocked like Z (padded to a multiple of bs, unit diagonal)
        z = Z.download()
        N = len(z.row_ptr) - 1
        D = np.eye(N * bs)
        m = min(N * bs, S.nb * 64)
        D[:m, :m] = dense_padded(S)[:m, :m]
        resid = oracle.resid(oracle.from_dense(D, bs, S.n), oracle.Mat(z.n, bs, z.row_ptr, z.col_idx, z.val))
        assert resid <= 1e-9, (S.n, resid)
    ifac.set_schedule(ctx, -1)
