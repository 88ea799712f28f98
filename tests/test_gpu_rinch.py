"""GPU recursive inverse Cholesky (Algorithm 1) through the C ABI against
the CPU oracle: same recursion depth, products and multiplied block pairs,
factor within 1e-10 relative Frobenius; without truncation the exact
inverse Cholesky factor at a size the oracle does not reach (checked through
Z^T S Z = I and the block upper-triangular pattern)."""
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


def _rel(gpu_host, ref) -> float:
    a = oracle.Mat(gpu_host.n, gpu_host.bs, gpu_host.row_ptr, gpu_host.col_idx, gpu_host.val).to_dense()
    b = ref.to_dense()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind,n,bs,leaf,tau", [("chain", 4096, 32, 512, 1e-10), ("chain", 1000, 32, 256, 1e-10),
                                                ("cluster", 1024, 32, 128, 1e-10), ("cluster", 768, 64, 128, 1e-8),
                                                ("chain", 512, 16, 512, 1e-10), ("cluster", 1500, 32, 200, 0.0)])
def test_rinch_matches_oracle(ctx, kind, n, bs, leaf, tau):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs, seed=0) if kind == "chain" else synth.cluster_overlap(n, bs, seed=0)
    Z_ref, rep_ref = oracle.rinch(S, tau=tau, leaf_size=leaf)
    Z, rep = ifac.inv_factor_rinch(ctx, ifac.upload(ctx, S), tau, ifac.opts(leaf_size=leaf))
    assert rep.levels == rep_ref.levels
    assert rep.products == rep_ref.products and rep.block_pairs == rep_ref.block_pairs
    zh = Z.download()
    assert _rel(zh, Z_ref) <= 1e-10
    assert np.array_equal(zh.row_ptr, Z_ref.row_ptr) and np.array_equal(zh.col_idx, Z_ref.col_idx)


def test_rinch_exact_factor_large(ctx):
    """tau = 0 on the 16,384-row chain (bs 32, 512-row leaves, 5 levels):
    block upper triangular and Z^T S Z = I to rounding."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(16384, 32, seed=7)
    dS = ifac.upload(ctx, S)
    Z, rep = ifac.inv_factor_rinch(ctx, dS, 0.0, ifac.opts(leaf_size=512))
    assert rep.levels == 5
    zh = Z.download()
    for I in range(zh.row_ptr.shape[0] - 1):
        cols = zh.col_idx[zh.row_ptr[I]:zh.row_ptr[I + 1]]
        assert cols[0] == I and np.all(np.diff(cols) > 0)
    assert ifac.inv_factor_resid(ctx, dS, Z) < 1e-11


def test_rinch_split_products(ctx):
    """Every product on the split tensor-core kernel (bs 64)."""
    from paper_1901_07993_gb300 import ifac
    S = synth.cluster_overlap(1024, 64, seed=3)
    Z_ref, rep_ref = oracle.rinch(S, tau=1e-10, leaf_size=128)
    Z, rep = ifac.inv_factor_rinch(ctx, ifac.upload(ctx, S), 1e-10, ifac.opts(leaf_size=128, prec=3))
    assert rep.split_pairs == rep.block_pairs > 0
    assert _rel(Z.download(), Z_ref) <= 1e-9


def test_rinch_not_spd(ctx):
    """A Schur complement that is not positive definite is reported."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(512, 32, seed=1)
    v = S.val.copy()
    last = S.row_ptr[-1] - 1  # the last diagonal block
    v[last] = -np.eye(32)
    bad = synth.HostBSR(S.n, S.bs, S.row_ptr, S.col_idx, v)
    with pytest.raises(ifac.IfacError) as ei:
        ifac.inv_factor_rinch(ctx, ifac.upload(ctx, bad), 0.0, ifac.opts(leaf_size=128))
    assert ei.value.code == ifac.ERR_NOT_SPD


@pytest.mark.parametrize("kind,n,bs,leaf,rrows", [("chain", 4096, 32, 128, 1024), ("cluster", 1024, 32, 64, 256)])
def test_lif_switch_to_rinch_matches_oracle(ctx, kind, n, bs, leaf, rrows):
    """LIF whose sub-problems of at most rrows rows are factorized by RINCH."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs, seed=2) if kind == "chain" else synth.cluster_overlap(n, bs, seed=2)
    Z_ref, rep_ref = oracle.lif(S, tau=1e-10, target=1e-10, leaf_size=leaf, rinch_rows=rrows)
    Z, rep = ifac.inv_factor_localized(ctx, ifac.upload(ctx, S), 1e-10, 1e-10,
                                       ifac.opts(leaf_size=leaf, rinch_rows=rrows))
    assert rep.levels == rep_ref.levels and rep.sweeps == rep_ref.sweeps
    assert rep.block_pairs == rep_ref.block_pairs
    assert _rel(Z.download(), Z_ref) <= 1e-10
