"""Pins for the oracle's refinement (IRSI) and localized inverse factorization.

IRSI (Section 2.2, Eq. 2.1): from Z_0 = c I every iterate is a polynomial in S,
so with S = V diag(lambda) V^T, Z_k = V diag(z_k(lambda)) V^T with the scalar
recurrence d = 1 - lambda z^2, z' = z sum_k b_k d^k.  Its limit is S^-1/2.

LIF (Algorithm 2): refinement from Z_0 keeps Z_i = Z_0 g_i(X) with
X = Z_0^T S Z_0, so each level converges to Z_0 (Z_0^T S Z_0)^-1/2, with the
leaves L^-T; a dense recursion built from numpy's eigh and cholesky gives the
expected factor.
"""
from math import comb

import numpy as np
import pytest

from paper_1901_07993_gb300 import synth


def _b(k):
    return comb(2 * k, k) / 4 ** k


def _closed_form_irsi(S, iters, m, c):
    w, V = np.linalg.eigh(S)
    z = np.full_like(w, c)
    deltas = []
    for _ in range(iters):
        d = 1 - w * z * z
        deltas.append(np.sqrt((d ** 2).sum()))
        z = z * sum(_b(k) * d ** k for k in range(m + 1))
    d = 1 - w * z * z
    deltas.append(np.sqrt((d ** 2).sum()))
    return (V * z) @ V.T, deltas


@pytest.mark.parametrize("m", [2, 4])
@pytest.mark.parametrize("c_rule", [0, 1])
def test_irsi_matches_eigen_recurrence(oracle_mod, m, c_rule):
    S = synth.chain_overlap(256, 32, seed=2)
    Sd = S.to_dense()
    beta = np.abs(Sd).sum(axis=1).max()
    c = 1 / np.sqrt(beta) if c_rule == 0 else np.sqrt(2 / beta)
    for k in (0, 1, 3):
        Z, rep = oracle_mod.irsi(S, m=m, tau=0.0, fixed_iters=k if k else 0, max_iter=0 if k == 0 else 50,
                                 c_rule=c_rule)
        Zc, deltas = _closed_form_irsi(Sd, k, m, c)
        assert rep.sweeps == k
        assert abs(rep.beta - beta) < 1e-13
        err = np.linalg.norm(Z.to_dense() - Zc) / np.linalg.norm(Zc)
        assert err < 1e-13, (k, err)
        assert np.allclose(rep.delta_fro[: k + 1], deltas, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("m", [2, 4])
def test_irsi_local_delta_matches_eigen_recurrence(oracle_mod, m):
    """Without truncation the local update of Eq. (2.2) is exact, so the
    locally updated delta norms and iterates follow the same closed form."""
    S = synth.cluster_overlap(256, 32, seed=3)
    Sd = S.to_dense()
    c = 1 / np.sqrt(np.abs(Sd).sum(axis=1).max())
    for k in (1, 4):
        Z, rep = oracle_mod.irsi(S, m=m, tau=0.0, fixed_iters=k, local_delta=True)
        Zc, deltas = _closed_form_irsi(Sd, k, m, c)
        assert rep.sweeps == k
        assert np.linalg.norm(Z.to_dense() - Zc) / np.linalg.norm(Zc) < 1e-12
        assert np.allclose(rep.delta_fro[: k + 1], deltas, rtol=1e-8, atol=1e-12)
        # local delta costs 3 more products per sweep than the 2 of a direct delta
        assert rep.products == 2 + k * (1 + (m - 1) + 3)


def test_irsi_converges_to_inverse_sqrt(oracle_mod):
    S = synth.chain_overlap(256, 32, seed=4)
    Sd = S.to_dense()
    Z, rep = oracle_mod.irsi(S, m=2, tau=0.0, target=0.0)
    w, V = np.linalg.eigh(Sd)
    Zs = (V / np.sqrt(w)) @ V.T
    assert rep.stop_reason == oracle_mod.STOP_RULE
    assert np.linalg.norm(Z.to_dense() - Zs) / np.linalg.norm(Zs) < 1e-13
    # cubic convergence of the tail (m = 2): e_{i+1} <~ C e_i^3
    e = rep.delta_fro
    i = next(k for k in range(len(e)) if e[k] < 0.2)
    assert e[i + 1] < 2 * e[i] ** 3 + 1e-13
    # symmetric iterates
    Zd = Z.to_dense()
    assert np.linalg.norm(Zd - Zd.T) < 1e-13


def test_irsi_stop_rule_returns_last_iterate(oracle_mod):
    S = synth.chain_overlap(256, 32, seed=4)
    Z, rep = oracle_mod.irsi(S, m=2, tau=1e-10, target=0.0)
    e = rep.delta_fro
    assert rep.stop_reason == oracle_mod.STOP_RULE
    # the rule fired on the last evaluation and on no earlier one
    assert e[-1] > e[-2] ** 3
    assert all(not (e[k] > e[k - 1] ** 3) for k in range(1, len(e) - 1))
    assert rep.sweeps == len(e) - 1
    # the returned Z is the one whose delta was evaluated last: recompute
    # delta = I - trunc(Z^T trunc(S_t Z)) with the same truncated products
    St = oracle_mod.truncate(S, 1e-10)
    X = oracle_mod.gemm(St, Z, tau=1e-10)
    Y = oracle_mod.gemm(Z, X, trans_a=True, tau=1e-10)
    assert oracle_mod.fro(oracle_mod.add(-1.0, Y, gamma=1.0)) == e[-1]
    # untruncated residual: at the truncation floor
    assert oracle_mod.resid(St, Z) < 1e-9
    # target stop
    Z2, rep2 = oracle_mod.irsi(S, m=2, tau=1e-10, target=1e-3)
    assert rep2.stop_reason == oracle_mod.STOP_TARGET and rep2.delta_fro[-1] <= 1e-3 < rep2.delta_fro[-2]


def _lif_dense(Sd, b0, b1, bs, leaf):
    nbs = b1 - b0
    Ss = Sd[b0 * bs:b1 * bs, b0 * bs:b1 * bs]
    if nbs * bs <= leaf or nbs == 1:
        return np.linalg.inv(np.linalg.cholesky(Ss)).T
    bm = b0 + nbs // 2
    ZA = _lif_dense(Sd, b0, bm, bs, leaf)
    ZC = _lif_dense(Sd, bm, b1, bs, leaf)
    Z0 = np.zeros_like(Ss)
    na = (bm - b0) * bs
    Z0[:na, :na] = ZA
    Z0[na:, na:] = ZC
    w, V = np.linalg.eigh(Z0.T @ Ss @ Z0)
    return Z0 @ ((V / np.sqrt(w)) @ V.T)


@pytest.mark.parametrize("kind,n,bs,leaf", [("chain", 256, 16, 64), ("chain", 200, 16, 48), ("cluster", 512, 32, 128)])
def test_lif_matches_dense_recursion(oracle_mod, kind, n, bs, leaf):
    S = synth.chain_overlap(n, bs, seed=1) if kind == "chain" else synth.cluster_overlap(n, bs, seed=1)
    Sd = S.to_dense()
    Z, rep = oracle_mod.lif(S, m=2, tau=0.0, target=0.0, leaf_size=leaf)
    Zr = _lif_dense(Sd, 0, S.nb, bs, leaf)
    err = np.linalg.norm(Z.to_dense() - Zr) / np.linalg.norm(Zr)
    assert err < 1e-11, err
    assert rep.status == 0 and rep.levels >= 2
    assert oracle_mod.resid(S, Z) < 1e-11


def test_lif_local_update_equals_direct_delta(oracle_mod):
    """First top-level sweep: the tracked delta_1 of Eq. (2.2) equals
    I - Z_1^T S Z_1 computed directly, with Z_1 = Z_0 (I + b1 delta_0 + b2 delta_0^2)."""
    n, bs, leaf = 256, 16, 128
    S = synth.chain_overlap(n, bs, seed=7)
    Sd = S.to_dense()
    Z, rep = oracle_mod.lif(S, m=2, tau=0.0, target=0.0, leaf_size=leaf)
    # top level children are leaves here (128 rows each)
    h = n // 2
    Z0 = np.zeros((n, n))
    Z0[:h, :h] = np.linalg.inv(np.linalg.cholesky(Sd[:h, :h])).T
    Z0[h:, h:] = np.linalg.inv(np.linalg.cholesky(Sd[h:, h:])).T
    d0 = np.eye(n) - Z0.T @ Sd @ Z0
    # the paper's bound on the start: ||delta_0||_2 <= 1 - lmin/lmax
    w = np.linalg.eigvalsh(Sd)
    assert np.linalg.norm(d0, 2) <= 1 - w[0] / w[-1] + 1e-12
    Z1 = Z0 @ (np.eye(n) + 0.5 * d0 + 0.375 * d0 @ d0)
    d1 = np.linalg.norm(np.eye(n) - Z1.T @ Sd @ Z1)
    assert abs(rep.delta_fro[0] - d1) <= 1e-10 * max(d1, 1e-3)


def test_lif_sweeps_within_iteration_bound(oracle_mod):
    """Sweep count per level <= K_max of Section 3.3 (plus the stop-rule check
    sweep), with eps at the reached accuracy."""
    S = synth.chain_overlap(256, 16, seed=3)
    Sd = S.to_dense()
    w = np.linalg.eigvalsh(Sd)
    Z, rep = oracle_mod.lif(S, m=2, tau=0.0, leaf_size=128)
    eps = 1e-14
    kmax = int(np.ceil(np.log(np.log(eps) / np.log(1 - w[0] / w[-1])) / np.log(3)))
    top = len(rep.delta_fro)
    assert top <= kmax + 2
