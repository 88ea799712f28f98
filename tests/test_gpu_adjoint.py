"""GPU adjoint of the refinement on a frozen block pattern (config: 1D chain,
bs 32, F = N(0,1) * S_ij symmetric on S's pattern, 6 sweeps) against the
oracle's adjoint (all entries, n = 512), against FP64 central differences
of the oracle's frozen-pattern loss (12 random stored entries at n = 16384:
each oracle forward takes seconds at that size), against FP64 central
differences of the library's own forward loss on 200 random stored entries
at n = 16384 (the forward loss itself is checked against the oracle's to
1e-12; 400 forwards take about 15 s), and the torch.autograd.Function
wrapper."""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
TAU, K = 1e-10, 6


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac.Context()


def _oracle_tape(S, F):
    c = 1.0 / np.sqrt(oracle.gershgorin(oracle.truncate(S, TAU)))
    tape = oracle.Tape(S, c, K, TAU)
    return tape, oracle.Mat(F.n, F.bs, F.row_ptr, F.col_idx, F.val)


def _on_pattern(G, S):
    """oracle gradient (truncated pattern) placed on S's pattern"""
    blocks = G.blocks()
    rows = np.repeat(np.arange(S.nb), np.diff(S.row_ptr))
    return np.array([blocks.get((int(i), int(j)), np.zeros((S.bs, S.bs))) for i, j in zip(rows, S.col_idx)])


def test_adjoint_matches_oracle_n512(ctx):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(512, 32, seed=0)
    F = synth.fock_like(S, seed=5)
    tape, Fo = _oracle_tape(S, F)
    L_ref = tape.loss(Fo)
    G_ref = _on_pattern(tape.adjoint(Fo), S)
    L, G = ifac.inv_factor_refine_adjoint(ctx, ifac.upload(ctx, S), ifac.upload(ctx, F), K, TAU)
    g = G.download()
    assert np.array_equal(g.col_idx, S.col_idx)
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    rel = np.linalg.norm(g.val - G_ref) / np.linalg.norm(G_ref)
    assert rel <= 1e-10, rel


def test_adjoint_central_differences_n16384(ctx):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(16384, 32, seed=0)
    F = synth.fock_like(S, seed=5)
    L, G = ifac.inv_factor_refine_adjoint(ctx, ifac.upload(ctx, S), ifac.upload(ctx, F), K, TAU)
    g = G.download()
    tape, Fo = _oracle_tape(S, F)
    St = tape.S()
    assert abs(L - tape.loss(Fo)) <= 1e-12 * abs(L)
    pos = {(int(i), int(j)): p for p, (i, j) in
           enumerate(zip(np.repeat(np.arange(S.nb), np.diff(S.row_ptr)), S.col_idx))}
    rows_t = np.repeat(np.arange(St.nb), np.diff(St.row_ptr))
    rng = np.random.default_rng(11)
    picks = rng.integers(0, St.nnzb, size=12)
    worst = 0.0
    for q in picks:
        r, s = rng.integers(0, 32, size=2)
        h = 1e-6 * max(1.0, abs(St.val[q, r, s]))
        Sp = oracle.Mat(St.n, 32, St.row_ptr, St.col_idx, St.val.copy())
        Sm = oracle.Mat(St.n, 32, St.row_ptr, St.col_idx, St.val.copy())
        Sp.val[q, r, s] += h
        Sm.val[q, r, s] -= h
        fd = (tape.frozen_loss(Sp, Fo) - tape.frozen_loss(Sm, Fo)) / (2 * h)
        p = pos[(int(rows_t[q]), int(St.col_idx[q]))]
        err = abs(fd - g.val[p, r, s]) / max(1.0, abs(fd))
        worst = max(worst, err)
    assert worst <= 1e-5, worst


def test_adjoint_central_differences_200_entries_n16384(ctx):
    """Config-5 size: dL/dS on 200 random stored entries (of S's pattern)
    against central differences h = 1e-4 max(1, |S_ij|) of the FP64 loss
    L(S +- h e_ij) that the library's forward pass returns.  Each forward
    re-records its block pattern by truncation at tau and sums in its own
    order, so L carries noise of about 1e-16 |L| and a jump where a block
    norm crosses tau; the larger step keeps both far below the tolerance
    (the truncation error of the difference is O(h^2))."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(16384, 32, seed=0)
    F = synth.fock_like(S, seed=5)
    dF = ifac.upload(ctx, F)
    L0, G = ifac.inv_factor_refine_adjoint(ctx, ifac.upload(ctx, S), dF, K, TAU)
    tape, Fo = _oracle_tape(S, F)
    assert abs(L0 - tape.loss(Fo)) <= 1e-12 * abs(L0)
    g = G.download()
    rng = np.random.default_rng(200)
    picks = rng.integers(0, S.nnzb, size=200)
    worst, errs = 0.0, []
    for q in picks:
        r, c = rng.integers(0, 32, size=2)
        h = 1e-4 * max(1.0, abs(S.val[q, r, c]))
        vals = []
        for sgn in (1.0, -1.0):
            v = S.val.copy()
            v[q, r, c] += sgn * h
            L, _ = ifac.inv_factor_refine_adjoint(ctx, ifac.upload(ctx, synth.HostBSR(S.n, 32, S.row_ptr,
                                                                                     S.col_idx, v)), dF, K, TAU)
            vals.append(L)
        fd = (vals[0] - vals[1]) / (2 * h)
        err = abs(fd - g.val[q, r, c]) / max(1.0, abs(fd))
        worst = max(worst, err)
        errs.append(err)
    print(f"200 entries: worst relative FD error {worst:.2e}, median {np.median(errs):.2e}, |L| {abs(L0):.3e}")
    assert worst <= 1e-5, worst


def test_autograd_function(ctx):
    import torch
    from paper_1901_07993_gb300 import ifac
    from paper_1901_07993_gb300.autograd import RefineLoss
    S = synth.chain_overlap(512, 32, seed=1)
    F = synth.fock_like(S, seed=5)
    val = torch.tensor(S.val, device="cuda", requires_grad=True)
    rp = torch.tensor(S.row_ptr, device="cuda")
    ci = torch.tensor(S.col_idx, device="cuda")
    dF = ifac.upload(ctx, F)
    L = RefineLoss.apply(val, rp, ci, S.n, 32, dF, K, TAU, ctx)
    (2.0 * L).backward()
    _, G = ifac.inv_factor_refine_adjoint(ctx, ifac.upload(ctx, S), dF, K, TAU)
    assert torch.allclose(val.grad.cpu(), 2.0 * torch.tensor(G.download().val), rtol=0, atol=0)
