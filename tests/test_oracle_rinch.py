"""Pins for the oracle's recursive inverse Cholesky (RINCH, Algorithm 1).

Without truncation RINCH computes the inverse Cholesky factor exactly: Z is
block upper triangular, the diagonal leaves are upper triangular with a
positive diagonal, and Z^T S Z = I, and the only matrix with those properties
is Z = L^-T for S = L L^T.  So at tau = 0 the oracle must equal numpy's
Cholesky-based inverse factor, whatever the leaf size and recursion depth.
With truncation the factor stays block upper triangular and Z^T S Z = I holds
to the truncation level."""
import numpy as np
import pytest

from paper_1901_07993_gb300 import synth


def _dense(m):
    return m.to_dense()


def _levels(nbs, bs, leaf):
    """Depth of the recursion: split at the block-aligned midpoint while a
    range has more than leaf rows and more than one block."""
    if nbs * bs <= leaf or nbs == 1:
        return 0
    h = nbs // 2
    return 1 + max(_levels(h, bs, leaf), _levels(nbs - h, bs, leaf))


def _inv_chol_factor(S):
    L = np.linalg.cholesky(S)
    return np.linalg.inv(L).T


@pytest.mark.parametrize("kind,n,bs,leaf", [("chain", 1000, 32, 128), ("chain", 640, 16, 64),
                                             ("cluster", 512, 32, 64), ("cluster", 777, 32, 96),
                                             ("chain", 300, 32, 4096)])
def test_rinch_is_the_inverse_cholesky_factor(oracle_mod, kind, n, bs, leaf):
    S = synth.chain_overlap(n, bs, seed=3) if kind == "chain" else synth.cluster_overlap(n, bs, seed=4)
    Z, rep = oracle_mod.rinch(S, tau=0.0, leaf_size=leaf)
    assert rep.status == 0
    Sd = oracle_mod.Mat(S.n, S.bs, S.row_ptr, S.col_idx, S.val).to_dense()
    Zd = _dense(Z)
    want = _inv_chol_factor(Sd)
    assert np.abs(Zd - want).max() <= 1e-11 * np.abs(want).max()
    assert np.allclose(np.triu(Zd), Zd, rtol=0, atol=0)
    assert rep.levels == _levels(-(-n // bs), bs, leaf)


@pytest.mark.parametrize("tau", [1e-10, 1e-6])
def test_rinch_truncated_keeps_structure(oracle_mod, tau):
    S = synth.cluster_overlap(1024, 32, seed=5)
    Z, rep = oracle_mod.rinch(S, tau=tau, leaf_size=128)
    for I in range(Z.nb):
        cols = Z.col_idx[Z.row_ptr[I]:Z.row_ptr[I + 1]]
        assert np.all(cols >= I) and (len(cols) and cols[0] == I)
    norms = np.sqrt((Z.val ** 2).sum(axis=(1, 2)))
    assert np.all(norms >= tau)
    r = oracle_mod.resid(S, Z)
    assert r <= 1e3 * tau
    assert rep.products == 4 * 7  # 4 products at each of the 7 internal nodes (1024 rows, 128-row leaves)


def test_rinch_single_leaf_is_the_leaf_routine(oracle_mod):
    S = synth.chain_overlap(256, 32, seed=6)
    Z, rep = oracle_mod.rinch(S, tau=0.0, leaf_size=256)
    Sd = oracle_mod.Mat(S.n, S.bs, S.row_ptr, S.col_idx, S.val).to_dense()
    assert rep.levels == 0 and rep.products == 0
    assert np.array_equal(_dense(Z), oracle_mod.invchol(Sd))


def test_lif_switch_to_rinch_equals_larger_leaves(oracle_mod):
    """Without truncation RINCH on a range returns that range's inverse
    Cholesky factor, which is what the dense leaf routine returns; so LIF
    switching to RINCH at R rows equals LIF with R-row dense leaves."""
    S = synth.cluster_overlap(512, 16, seed=8)
    Za, ra = oracle_mod.lif(S, tau=0.0, target=1e-12, leaf_size=32, rinch_rows=128)
    Zb, rb = oracle_mod.lif(S, tau=0.0, target=1e-12, leaf_size=128)
    assert ra.levels == rb.levels
    za, zb = Za.to_dense(), Zb.to_dense()
    assert np.abs(za - zb).max() <= 1e-10 * np.abs(zb).max()
    r_more = oracle_mod.lif(S, tau=0.0, target=1e-12, leaf_size=32)[1]
    assert r_more.levels > ra.levels
