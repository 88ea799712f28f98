"""Pins of the oracle's adjoint of the refinement on a frozen block pattern:
central finite differences of the frozen-pattern loss L = tr(Z_K^T F Z_K) on
single entries of S (all entries independent) and on symmetric pairs; the
recording run and the frozen forward agree; with no sweep L does not depend
on S."""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth


def _setup(n=160, bs=16, K=3, tau=1e-9, seed=2):
    S = synth.chain_overlap(n, bs, seed=seed)
    F = synth.fock_like(S, seed=5)
    beta = oracle.gershgorin(oracle.truncate(S, tau))
    c = 1.0 / np.sqrt(beta)
    tape = oracle.Tape(S, c, K, tau)
    St = tape.S()
    Ft = oracle.Mat(F.n, bs, F.row_ptr, F.col_idx, F.val)
    return S, St, Ft, tape, c


def test_frozen_forward_reproduces_recording():
    S, St, F, tape, c = _setup()
    L_rec = tape.loss(F)
    L_frz = tape.frozen_loss(St, F)
    assert abs(L_rec - L_frz) <= 1e-13 * abs(L_rec)


def test_no_sweep_no_dependence():
    S = synth.chain_overlap(64, 16, seed=1)
    F = synth.fock_like(S, seed=5)
    tape = oracle.Tape(S, 0.7, 0, 1e-9)
    G = tape.adjoint(oracle.Mat(F.n, 16, F.row_ptr, F.col_idx, F.val))
    assert np.all(G.val == 0)
    assert abs(tape.loss(oracle.Mat(F.n, 16, F.row_ptr, F.col_idx, F.val)) - 0.49 * np.trace(F.to_dense())) < 1e-12


@pytest.mark.parametrize("K", [1, 3])
def test_adjoint_matches_central_differences(K):
    S, St, F, tape, c = _setup(K=K)
    G = tape.adjoint(F)
    assert np.array_equal(G.col_idx, St.col_idx)
    rng = np.random.default_rng(7)
    picks = rng.integers(0, St.nnzb, size=12)
    for p in picks:
        r, s = rng.integers(0, St.bs, size=2)
        h = 1e-6 * max(1.0, abs(St.val[p, r, s]))
        Sp = oracle.Mat(St.n, St.bs, St.row_ptr, St.col_idx, St.val.copy())
        Sm = oracle.Mat(St.n, St.bs, St.row_ptr, St.col_idx, St.val.copy())
        Sp.val[p, r, s] += h
        Sm.val[p, r, s] -= h
        fd = (tape.frozen_loss(Sp, F) - tape.frozen_loss(Sm, F)) / (2 * h)
        assert abs(fd - G.val[p, r, s]) <= 1e-6 * max(1.0, abs(fd)), (p, r, s, fd, G.val[p, r, s])


def test_adjoint_symmetric_direction():
    """Perturbing S_ij and S_ji together: derivative = G_ij + G_ji."""
    S, St, F, tape, c = _setup(K=2)
    G = tape.adjoint(F)
    Gd = G.to_dense()
    Sd = St.to_dense()
    i, j = 5, 21
    assert Sd[i, j] != 0
    h = 1e-6
    bs = St.bs

    def perturbed(sign):
        D = Sd.copy()
        D[i, j] += sign * h
        D[j, i] += sign * h
        v = np.array([D[a * bs:(a + 1) * bs, b * bs:(b + 1) * bs]
                      for a, b in zip(np.repeat(np.arange(St.nb), np.diff(St.row_ptr)), St.col_idx)])
        return oracle.Mat(St.n, bs, St.row_ptr, St.col_idx, v)

    fd = (tape.frozen_loss(perturbed(1), F) - tape.frozen_loss(perturbed(-1), F)) / (2 * h)
    assert abs(fd - (Gd[i, j] + Gd[j, i])) <= 1e-6 * max(1.0, abs(fd))
