"""GPU parity of the factorizations against the CPU oracle through the C ABI:
refinement from a scaled identity and localized inverse factorization, at the
1D-chain size of the benchmark (n = 4096, bs 32, tau = 1e-10) and on ragged
and 3D cases.  The bar is ||Z_gpu - Z_oracle||_F / ||Z_oracle||_F <= 1e-10
(missing blocks count as zero), equal sweep counts, and matching delta norms."""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac.Context()


def _rel(gpu_host, ref: oracle.Mat) -> float:
    a = oracle.Mat(gpu_host.n, gpu_host.bs, gpu_host.row_ptr, gpu_host.col_idx, gpu_host.val).to_dense()
    b = ref.to_dense()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,bs,tau,m", [(4096, 32, 1e-10, 2), (1000, 32, 1e-10, 2), (640, 16, 1e-8, 4),
                                        (2048, 64, 1e-12, 2)])
def test_refine_matches_oracle(ctx, n, bs, tau, m):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs, seed=0)
    Z_ref, rep_ref = oracle.irsi(S, m=m, tau=tau, target=1e-10)
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), tau, 1e-10, ifac.opts(m=m))
    assert rep.sweeps == rep_ref.sweeps and rep.stop_reason == rep_ref.stop_reason
    assert abs(rep.beta - rep_ref.beta) <= 1e-13 * rep_ref.beta
    assert np.allclose(rep.delta_fro, rep_ref.delta_fro, rtol=1e-6, atol=1e-12)
    assert _rel(Z.download(), Z_ref) <= TOL
    assert rep.products == rep_ref.products and rep.block_pairs == rep_ref.block_pairs


def test_refine_fixed_iterations_and_resid(ctx):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(1024, 32, seed=3)
    Z_ref, _ = oracle.irsi(S, tau=0.0, fixed_iters=3)
    dS = ifac.upload(ctx, S)
    Z, rep = ifac.inv_factor_refine(ctx, dS, 0.0, 0.0, ifac.opts(fixed_iters=3))
    assert rep.sweeps == 3 and rep.stop_reason == ifac.STOP_FIXED
    assert _rel(Z.download(), Z_ref) <= TOL
    r = ifac.inv_factor_resid(ctx, dS, Z)
    assert abs(r - oracle.resid(S, Z_ref)) <= 1e-9 * max(r, 1e-3)


@pytest.mark.parametrize("kind,n,bs,leaf,tau", [("chain", 4096, 32, 512, 1e-10), ("chain", 1000, 32, 256, 1e-10),
                                                ("cluster", 1024, 32, 256, 1e-10), ("cluster", 768, 64, 128, 1e-8),
                                                ("chain", 512, 16, 512, 1e-10)])
def test_localized_matches_oracle(ctx, kind, n, bs, leaf, tau):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs, seed=0) if kind == "chain" else synth.cluster_overlap(n, bs, seed=0)
    Z_ref, rep_ref = oracle.lif(S, tau=tau, target=1e-10, leaf_size=leaf)
    Z, rep = ifac.inv_factor_localized(ctx, ifac.upload(ctx, S), tau, 1e-10, ifac.opts(leaf_size=leaf))
    assert rep.levels == rep_ref.levels
    assert rep.sweeps == rep_ref.sweeps
    assert np.allclose(rep.delta_fro, rep_ref.delta_fro, rtol=1e-6, atol=1e-12)
    assert _rel(Z.download(), Z_ref) <= TOL
    # one batched product serves all sub-problems of a level, so only the
    # multiplied block pairs (not the product calls) must agree
    assert rep.block_pairs == rep_ref.block_pairs


def test_localized_zero_tau_invariant(ctx):
    """Z^T S Z = I holds at any size: n = 8192 chain, checked on the GPU."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(8192, 32, seed=5)
    dS = ifac.upload(ctx, S)
    Z, rep = ifac.inv_factor_localized(ctx, dS, 0.0, 0.0, ifac.opts(leaf_size=512))
    assert ifac.inv_factor_resid(ctx, dS, Z) < 1e-11


@pytest.mark.parametrize("kind,n,bs,tau,m", [("chain", 4096, 32, 1e-10, 2), ("cluster", 1024, 32, 1e-8, 4),
                                             ("chain", 2000, 32, 1e-5, 4)])
def test_refine_local_delta_matches_oracle(ctx, kind, n, bs, tau, m):
    """IRSI with the local delta update of Eq. (2.2), as in the paper's runs."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, bs, seed=0) if kind == "chain" else synth.cluster_overlap(n, bs, seed=0)
    Z_ref, rep_ref = oracle.irsi(S, m=m, tau=tau, target=1e-10, local_delta=True)
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), tau, 1e-10, ifac.opts(m=m, local_delta=True))
    assert rep.sweeps == rep_ref.sweeps and rep.stop_reason == rep_ref.stop_reason
    assert np.allclose(rep.delta_fro, rep_ref.delta_fro, rtol=1e-6, atol=1e-12)
    assert _rel(Z.download(), Z_ref) <= TOL
    assert rep.products == rep_ref.products and rep.block_pairs == rep_ref.block_pairs
