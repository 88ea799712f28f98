"""The mixed-precision refinement on config 3's 3D geometry (random
sequential addition at 0.1 points per bohr^3, RCB order, block-dense factor)
at n = 16,384, bs 64, tau = 1e-14, target 1e-10: TF32 sweeps, then delta
with split FP64-accurate products of 8 slices (Section 2.2, Eq. 2.1).

As for the full-size chain, the factor is S^-1/2 Q and the oracle cannot
refine a matrix of this size in a test, so properties are checked: the stop
at the target, the direct residual with FP64-pipe products, and the oracle's
own FP64 evaluation of the residual block delta_WW = I - (Z^T S Z)_WW from the
returned Z on three windows W of block columns, each bounded by the whole
residual (the window evaluation is pinned to the dense definition on CPU in
test_gpu_zfullsize.py)."""
import pytest

from paper_1901_07993_gb300 import synth
from test_gpu_zfullsize import window_residual

pytestmark = pytest.mark.gpu
N, BS, TAU, TARGET = 16384, 64, 1e-14, 1e-10


def test_mixed_3d_cluster_meets_target():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    ctx = ifac.Context()
    ctx.set_split_slices(8)
    S = synth.cluster_overlap(N, BS, seed=0)
    dS = ifac.upload(ctx, S)
    Z, rep = ifac.inv_factor_refine(ctx, dS, TAU, TARGET, ifac.opts(m=2, prec=1, max_iter=100))
    assert rep.stop_reason == ifac.STOP_TARGET
    assert rep.low_sweeps >= 2 and rep.fp64_delta_evals >= 1 and rep.split_launches > 0
    assert rep.delta_fro[-1] <= TARGET
    resid = ifac.inv_factor_resid(ctx, dS, Z)  # FP64-pipe products, untruncated
    assert resid <= TARGET
    Zh = Z.download()
    nb = Zh.nb
    assert Zh.nnzb > 0.9 * nb * nb  # block-dense factor
    worst = 0.0
    for a in (0, nb // 2, nb - 2):
        r = window_residual(S, Zh, a, a + 2)
        worst = max(worst, r)
        assert r <= resid + 1e-13
    print(f"3D n {N}: sweeps {rep.sweeps} ({rep.low_sweeps} low, {rep.fp64_delta_evals} split delta), "
          f"residual {resid:.3e}, largest sampled window residual {worst:.3e}, nnzb {Zh.nnzb}")
