"""GPU parity of the block-sparse operations against the CPU oracle, through
the C ABI: products with truncation (every transpose combination, ragged
sizes, empty rows, empty operands), sums, truncation, norms, Gershgorin and
the batched leaf inverse Cholesky."""
import itertools

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


def _ifac():
    from paper_1901_07993_gb300 import ifac
    return ifac


def _as_oracle(h):
    return oracle.Mat(h.n, h.bs, h.row_ptr, h.col_idx, h.val)


def _midpoint_tau(ref: oracle.Mat):
    norms = sorted(np.sqrt((ref.val ** 2).sum(axis=(1, 2))))
    if len(norms) < 2:
        return 0.0
    k = len(norms) // 2
    return 0.5 * (norms[k - 1] + norms[k])


@pytest.mark.parametrize("bs", [16, 32, 64])
@pytest.mark.parametrize("tA,tB", list(itertools.product([False, True], repeat=2)))
def test_gemm_trunc_matches_oracle(ctx, bs, tA, tB):
    ifac = _ifac()
    nb = 11
    A = synth.random_bsr(nb, bs, 0.35, seed=100 + bs, empty_rows=2, n=nb * bs - 5)
    B = synth.random_bsr(nb, bs, 0.35, seed=200 + bs, empty_rows=1, n=nb * bs - 5)
    dA, dB = ifac.upload(ctx, A), ifac.upload(ctx, B)
    ref0 = oracle.gemm(A, B, tA, tB, -0.75, 0.0)
    tau = _midpoint_tau(ref0)
    for t in (0.0, tau):
        ref = oracle.gemm(A, B, tA, tB, -0.75, t)
        got = ifac.bsr_gemm_trunc(ctx, dA, tA, dB, tB, -0.75, t).download()
        assert np.array_equal(got.row_ptr, ref.row_ptr)
        assert np.array_equal(got.col_idx, ref.col_idx)
        scale = np.abs(ref.val).max() if ref.nnzb else 1.0
        assert np.abs(got.val - ref.val).max() <= 1e-13 * scale


def test_gemm_empty_and_single_block(ctx):
    ifac = _ifac()
    E = synth.random_bsr(6, 32, 0.0, seed=1)
    F = synth.random_bsr(6, 32, 0.5, seed=2)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, E), False, ifac.upload(ctx, F), False).download()
    assert got.nnzb == 0 and np.all(got.row_ptr == 0)
    one = synth.random_bsr(1, 64, 1.0, seed=3)
    ref = oracle.gemm(one, one, True, False)
    got = ifac.bsr_gemm_trunc(ctx, ifac.upload(ctx, one), True, ifac.upload(ctx, one), False).download()
    assert np.allclose(got.val, ref.val, rtol=0, atol=1e-12 * np.abs(ref.val).max())


def test_gemm_overlap_products(ctx):
    """S Z and Z^T (S Z) shapes on the 1D chain at block size 32."""
    ifac = _ifac()
    S = synth.chain_overlap(4096, 32, seed=0)
    St = oracle.truncate(S, 1e-10)
    dS = ifac.bsr_truncate(ctx, ifac.upload(ctx, S), 1e-10)
    dSh = dS.download()
    assert np.array_equal(dSh.col_idx, St.col_idx) and np.array_equal(dSh.val, St.val)
    X_ref = oracle.gemm(St, St, False, False, 1.0, 1e-10)
    X = ifac.bsr_gemm_trunc(ctx, dS, False, dS, False, 1.0, 1e-10).download()
    assert np.array_equal(X.col_idx, X_ref.col_idx)
    assert np.abs(X.val - X_ref.val).max() <= 1e-14 * np.abs(X_ref.val).max()


def test_add_bitwise(ctx):
    ifac = _ifac()
    A = synth.random_bsr(9, 32, 0.3, seed=5)
    B = synth.random_bsr(9, 32, 0.3, seed=6)
    ref = oracle.add(0.5, A, -2.0, B, 1.5)
    got = ifac.bsr_add(ctx, 0.5, ifac.upload(ctx, A), -2.0, ifac.upload(ctx, B), 1.5).download()
    assert np.array_equal(got.col_idx, ref.col_idx)
    assert np.array_equal(got.val, ref.val)  # same operation order, no contraction
    ref2 = oracle.add(-1.0, A, gamma=1.0)
    got2 = ifac.bsr_add(ctx, -1.0, ifac.upload(ctx, A), 0.0, None, 1.0).download()
    assert np.array_equal(got2.val, ref2.val)


def test_fro_and_gershgorin(ctx):
    ifac = _ifac()
    S = synth.cluster_overlap(1024, 64, seed=0)
    dS = ifac.upload(ctx, S)
    assert abs(ifac.bsr_fro(ctx, dS) - oracle.fro(S)) <= 1e-13 * oracle.fro(S)
    assert abs(ifac.bsr_gershgorin(ctx, dS) - oracle.gershgorin(S)) <= 1e-13 * oracle.gershgorin(S)


@pytest.mark.parametrize("nl", [96, 128, 512, 200])
def test_leaf_invchol_batched(ctx, nl):
    import torch
    ifac = _ifac()
    mats = []
    for k in range(3):
        S = synth.cluster_overlap(nl, 32, seed=k).to_dense()[:nl, :nl] if nl % 32 == 0 else \
            synth.chain_overlap(nl, 8, seed=k).to_dense()[:nl, :nl]
        mats.append(S)
    St = torch.tensor(np.array(mats), device="cuda")
    Z, info, rc = ifac.leaf_invchol_batched(ctx, St)
    assert rc == 0 and int(info.abs().sum()) == 0
    Zh = Z.cpu().numpy()
    for k in range(3):
        ref = oracle.invchol(mats[k])
        assert np.array_equal(Zh[k], np.triu(Zh[k]))
        err = np.linalg.norm(Zh[k] - ref) / np.linalg.norm(ref)
        assert err < 1e-10, err


def test_leaf_invchol_reports_not_spd(ctx):
    import torch
    ifac = _ifac()
    S = synth.chain_overlap(64, 32, seed=1).to_dense()
    bad = S.copy()
    bad[40, 40] = -1.0
    St = torch.tensor(np.array([S, bad]), device="cuda")
    Z, info, rc = ifac.leaf_invchol_batched(ctx, St)
    assert rc == ifac.ERR_NOT_SPD
    assert int(info[0]) == 0 and int(info[1]) == 41


def test_upload_rejects_malformed(ctx):
    ifac = _ifac()
    A = synth.random_bsr(4, 16, 0.8, seed=9)
    bad = synth.HostBSR(A.n, A.bs, A.row_ptr.copy(), A.col_idx.copy(), A.val)
    r0 = bad.row_ptr[0]
    if bad.row_ptr[1] - r0 >= 2:
        bad.col_idx[r0], bad.col_idx[r0 + 1] = bad.col_idx[r0 + 1], bad.col_idx[r0]
    else:
        bad.col_idx[0] = 99
    with pytest.raises(ifac.IfacError) as e:
        ifac.upload(ctx, bad)
    assert e.value.code == ifac.ERR_INVALID
