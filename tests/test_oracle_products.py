"""Pins for the oracle's block-sparse primitives against brute force.

Each check expands the operands to dense, applies the definition with numpy,
and compares; truncation is checked as "dense product, then drop every output
block whose Frobenius norm is strictly below tau" (Section 5 of the paper).
"""
import itertools

import numpy as np
import pytest

from paper_1901_07993_gb300 import synth


def _dense_pattern(A, B, tA, tB):
    """(I, J) pairs for which some K has op(A)_IK and op(B)_KJ stored."""
    ma = np.zeros((A.nb, A.nb), bool)
    mb = np.zeros((B.nb, B.nb), bool)
    for M, m in ((A, ma), (B, mb)):
        rows = np.repeat(np.arange(M.nb), np.diff(M.row_ptr))
        m[rows, M.col_idx] = True
    if tA:
        ma = ma.T
    if tB:
        mb = mb.T
    return (ma.astype(int) @ mb.astype(int)) > 0


@pytest.mark.parametrize("bs,nb,dens,empty", [(1, 7, 0.4, 1), (3, 9, 0.3, 2), (8, 5, 1.0, 0), (4, 6, 0.0, 0)])
@pytest.mark.parametrize("tA,tB", list(itertools.product([False, True], repeat=2)))
def test_gemm_matches_dense(oracle_mod, bs, nb, dens, empty, tA, tB):
    A = synth.random_bsr(nb, bs, dens, seed=11, empty_rows=empty)
    B = synth.random_bsr(nb, bs, dens, seed=12, empty_rows=empty)
    alpha = -0.7
    Ad, Bd = A.to_dense(), B.to_dense()
    ref = alpha * ((Ad.T if tA else Ad) @ (Bd.T if tB else Bd))
    pat = _dense_pattern(A, B, tA, tB)
    C = oracle_mod.gemm(A, B, tA, tB, alpha, 0.0)
    assert np.allclose(C.to_dense(), ref, rtol=0, atol=1e-12)
    got = {k for k in C.blocks()}
    assert got == {(int(i), int(j)) for i, j in zip(*np.nonzero(pat))}
    # truncation: pick tau between block norms so a good part is dropped
    norms = sorted(np.linalg.norm(ref[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]) for i, j in zip(*np.nonzero(pat)))
    if len(norms) >= 2:
        k = len(norms) // 2
        tau = 0.5 * (norms[k - 1] + norms[k])  # between two norms: no rounding tie
        Ct = oracle_mod.gemm(A, B, tA, tB, alpha, tau)
        keep = {(int(i), int(j)) for i, j in zip(*np.nonzero(pat))
                if not (np.linalg.norm(ref[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]) < tau)}
        assert set(Ct.blocks()) == keep
        for (i, j), blk in Ct.blocks().items():
            assert np.allclose(blk, ref[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs], atol=1e-12)


def test_gemm_rows_sorted_and_counters(oracle_mod):
    A = synth.random_bsr(12, 2, 0.5, seed=3)
    C = oracle_mod.gemm(A, A, True, False)
    for i in range(C.nb):
        cols = C.col_idx[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_add_matches_dense(oracle_mod):
    A = synth.random_bsr(8, 3, 0.3, seed=5)
    B = synth.random_bsr(8, 3, 0.3, seed=6)
    C = oracle_mod.add(0.5, A, -2.0, B, 1.5)
    ref = 0.5 * A.to_dense() - 2.0 * B.to_dense() + 1.5 * np.eye(24)
    assert np.allclose(C.to_dense(), ref, atol=1e-14)
    # union pattern + diagonal
    pa = set(oracle_mod.Mat(A.n, 3, A.row_ptr, A.col_idx, A.val).blocks())
    pb = set(oracle_mod.Mat(B.n, 3, B.row_ptr, B.col_idx, B.val).blocks())
    assert set(C.blocks()) == pa | pb | {(i, i) for i in range(8)}
    C2 = oracle_mod.add(-1.0, A)
    assert set(C2.blocks()) == pa


def test_truncate_transpose_fro_gershgorin(oracle_mod):
    A = synth.random_bsr(9, 4, 0.5, seed=8)
    Ad = A.to_dense()
    norms = np.sqrt((A.val ** 2).sum(axis=(1, 2)))
    tau = np.median(norms)
    T = oracle_mod.truncate(A, tau)
    assert T.nnzb == int((norms >= tau).sum())
    assert np.array_equal(oracle_mod.transpose(A).to_dense(), Ad.T)
    assert abs(oracle_mod.fro(A) - np.linalg.norm(Ad)) <= 1e-12 * np.linalg.norm(Ad)
    assert abs(oracle_mod.gershgorin(A) - np.abs(Ad).sum(axis=1).max()) <= 1e-12


def test_refinement_coefficients(oracle_mod):
    # b_k = (2k-1)/(2k) b_{k-1}, b_0 = 1 has the closed form binom(2k, k) / 4^k
    from math import comb
    for k in range(0, 8):
        assert oracle_mod.coef_b(k) == comb(2 * k, k) / 4 ** k
    assert [oracle_mod.coef_b(k) for k in range(5)] == [1, 0.5, 0.375, 0.3125, 35 / 128]


def test_invchol_leaf(oracle_mod):
    S = synth.chain_overlap(96, 32).to_dense()
    Z = oracle_mod.invchol(S)
    L = np.linalg.cholesky(S)
    assert np.allclose(Z, np.linalg.inv(L).T, atol=1e-12)
    assert np.array_equal(Z, np.triu(Z)) and np.all(np.diag(Z) > 0)
    assert np.linalg.norm(np.eye(96) - Z.T @ S @ Z) < 1e-12
    bad = S.copy()
    bad[5, 5] = -1.0
    with pytest.raises(np.linalg.LinAlgError):
        oracle_mod.invchol(bad)


def test_resid(oracle_mod):
    S = synth.chain_overlap(128, 32)
    Sd = S.to_dense()
    w, V = np.linalg.eigh(Sd)
    Zd = (V / np.sqrt(w)) @ V.T
    Z = oracle_mod.from_dense(Zd, 32)
    assert oracle_mod.resid(S, Z) < 1e-12
    Z2 = oracle_mod.from_dense(0.9 * Zd, 32)
    assert abs(oracle_mod.resid(S, Z2) - np.linalg.norm(np.eye(128) - 0.81 * np.eye(128))) < 1e-10
