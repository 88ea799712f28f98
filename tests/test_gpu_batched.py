"""Batched refinement: independent matrices refined together (block-diagonal
batching, per-member stop tests) through the C ABI.  In FP64 every member must
match the oracle's refinement of that member alone (same sweep count, factor
within 1e-10 relative Frobenius); with TF32/BF16 products every member
follows the mixed-precision schedule (low-precision sweeps, then delta with
FP64-accurate split products) and must reach its FP64 floor or the target;
the reported residual is checked against the oracle's residual of the
returned factor."""
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


def _members(bs):
    return [synth.chain_overlap(700, bs, seed=1), synth.cluster_overlap(512, bs, seed=2),
            synth.chain_overlap(2600, bs, seed=3), synth.cluster_overlap(1000, bs, seed=4),
            synth.chain_overlap(1500, bs, seed=5)]


def _dense(h):
    return oracle.Mat(h.n, h.bs, h.row_ptr, h.col_idx, h.val).to_dense()


@pytest.mark.parametrize("bs", [32, 64])
def test_batched_fp64_matches_members(ctx, bs):
    from paper_1901_07993_gb300 import ifac
    Ss = _members(bs)
    dS = [ifac.upload(ctx, S) for S in Ss]
    Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, 1e-10, 1e-10, ifac.opts())
    for S, Z, rep in zip(Ss, Zs, reps):
        Z_ref, rep_ref = oracle.irsi(S, tau=1e-10, target=1e-10)
        assert rep.sweeps == rep_ref.sweeps and rep.stop_reason == rep_ref.stop_reason
        assert np.allclose(rep.delta_fro, rep_ref.delta_fro, rtol=1e-6, atol=1e-12)
        zr = Z_ref.to_dense()
        assert np.linalg.norm(_dense(Z.download()) - zr) / np.linalg.norm(zr) <= 1e-10
        assert abs(rep.resid_fro - oracle.resid(oracle.truncate(S, 1e-10), Z_ref)) <= 1e-9


@pytest.mark.parametrize("prec", [1, 2])
def test_batched_low_precision(ctx, prec):
    """tau = 1e-10: the truncation floor (about 1e-9) sits above the 1e-10
    target, so members stop when ||delta||_F stops falling in the FP64 phase."""
    from paper_1901_07993_gb300 import ifac
    Ss = _members(64)
    dS = [ifac.upload(ctx, S) for S in Ss]
    Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, 1e-10, 1e-10, ifac.opts(prec=prec))
    for S, Z, rep in zip(Ss, Zs, reps):
        print(f"n={S.n} prec={prec}: sweeps {rep.sweeps} ({rep.low_sweeps} low, {rep.fp64_delta_evals} FP64 delta), "
              f"residual {rep.resid_fro:.3e}, delta {['%.3g' % e for e in rep.delta_fro]}")
        assert rep.stop_reason in (1, 2) and rep.low_sweeps >= 2 and rep.fp64_delta_evals >= 1
        assert rep.resid_fro <= 1e-8
        assert rep.tc_pairs > 0 and rep.split_pairs > 0


@pytest.mark.parametrize("prec", [1, 2])
def test_batched_mixed_meets_target(ctx, prec):
    """tau = 1e-12: every member reaches the 1e-10 target; the reported
    residual (split FP64-accurate products) agrees with the oracle's FP64
    residual of the returned factor."""
    from paper_1901_07993_gb300 import ifac
    Ss = _members(64)
    dS = [ifac.upload(ctx, S) for S in Ss]
    Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=prec))
    assert rc == ifac.OK
    for S, Z, rep in zip(Ss, Zs, reps):
        assert rep.stop_reason == ifac.STOP_TARGET and rep.fp64_delta_evals >= 1
        zh = Z.download()
        r_ref = oracle.resid(S, oracle.Mat(zh.n, zh.bs, zh.row_ptr, zh.col_idx, zh.val))
        assert r_ref <= 1e-10
        assert abs(rep.resid_fro - r_ref) <= 1e-11 + 1e-3 * r_ref
