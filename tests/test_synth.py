"""Input generator: published RNG vector, geometry constraints, overlap matrix
properties (S_ii = 1, symmetry, positive definiteness, the Gaussian formula)."""
import numpy as np

from paper_1901_07993_gb300 import synth


def test_splitmix64_reference_vector():
    # SplitMix64 seeded with 0: the first three outputs of the published
    # reference implementation (Steele, Lea, Flood 2014; Vigna's splitmix64.c).
    assert synth.rng_draw(0, 1) == 0xE220A8397B1DCDAF
    assert synth.rng_draw(0, 2) == 0x6E789E6AA1B965F4
    assert synth.rng_draw(0, 3) == 0x06C45D188009454F


def test_chain_geometry():
    g = synth.chain(500, seed=0)
    x = g.xyz[:, 0]
    off = x - 1.4 * np.arange(500)
    assert np.all(np.abs(off) <= 0.1) and off.std() > 0.04
    assert np.all(g.xyz[:, 1:] == 0)
    assert list(g.alpha[:4]) == [0.17, 0.62, 3.4, 0.17]


def test_cluster_geometry_and_rcb():
    n, bs = 1024, 32
    g = synth.cluster(n, bs, seed=0)
    L = (n / 0.1) ** (1 / 3)
    assert np.all(g.xyz >= 0) and np.all(g.xyz < L)
    d2 = ((g.xyz[:, None, :] - g.xyz[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 1.8 ** 2
    # exponents are a permutation of the cyclic assignment
    assert sorted(g.alpha) == sorted(synth.exponents(n))
    # RCB: the two halves are separated along one axis
    a, b = g.xyz[: n // 2], g.xyz[n // 2:]
    assert any(a[:, c].max() <= b[:, c].min() or b[:, c].max() <= a[:, c].min() for c in range(3))


def test_overlap_matrix_properties():
    g = synth.chain(200, seed=1)
    S = synth.overlap_bsr(g, 16)  # 200 = 12.5 blocks -> padded last block
    assert S.nb == 13
    D = S.to_dense()
    assert np.array_equal(np.diag(D), np.ones(208))
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    # the formula, at one pair
    i, j = 3, 5
    a, b = g.alpha[i], g.alpha[j]
    r2 = ((g.xyz[i] - g.xyz[j]) ** 2).sum()
    ref = (2 * np.sqrt(a * b) / (a + b)) ** 1.5 * np.exp(-a * b / (a + b) * r2)
    assert abs(D[i, j] - ref) <= 1e-15
    # padding rows are identity
    assert np.array_equal(D[200:, :200], np.zeros((8, 200)))


def test_generation_cutoff_is_far_below_tau():
    g = synth.cluster(512, 32, seed=0)
    S = synth.overlap_bsr(g, 32)
    norms = np.sqrt((S.val ** 2).sum(axis=(1, 2)))
    assert norms.min() >= synth.GEN_DROP
