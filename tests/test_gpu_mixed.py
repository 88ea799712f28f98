"""Mixed-precision refinement (TF32 / BF16 tensor-core products, FP64 sums,
norms and final delta evaluations) through the C ABI.  It has no pin beyond
the FP64 oracle: the refinement from a scaled identity converges to the same
S^-1/2 whatever the precision of the corrections, so the result is compared
with the oracle's FP64 factor, and the error is stated; the direct FP64
residual ||I - Z^T S Z||_F must reach the target.  With low-precision
corrections the iterates leave the polynomials in S, so Z converges to another
inverse factor S^-1/2 Q (Q near orthogonal): its distance to the FP64 factor is
stated, and bounded by three times the distance measured on GB300 for each
case (chain n = 4096: TF32 7.0e-5, BF16 5.5e-4; 3D cluster n = 1024: TF32
7.2e-4, BF16 5.5e-3), so that a change in the low-precision products shows.
The residual is the oracle's FP64 ||I - Z^T S Z||_F of the downloaded factor,
not the library's own."""
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


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("kind,n", [("chain", 4096), ("cluster", 1024)])
def test_mixed_refine_reaches_target(ctx, prec, kind, n):
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(n, 64, seed=0) if kind == "chain" else synth.cluster_overlap(n, 64, seed=0)
    tau, target = 1e-13, 1e-10
    dS = ifac.upload(ctx, S)
    Z, rep = ifac.inv_factor_refine(ctx, dS, tau, target, ifac.opts(prec=prec, max_iter=80))
    a = Z.download()
    Zh = oracle.Mat(a.n, 64, a.row_ptr, a.col_idx, a.val)
    resid = oracle.resid(S, Zh)
    resid_gpu = ifac.inv_factor_resid(ctx, dS, Z)
    Z_ref, rep_ref = oracle.irsi(S, tau=tau, target=target, max_iter=80)
    za = Zh.to_dense()
    zr = Z_ref.to_dense()
    rel = np.linalg.norm(za - zr) / np.linalg.norm(zr)
    print(f"{kind} n={n} prec={prec}: resid {resid:.2e} (library {resid_gpu:.2e}), rel err vs FP64 oracle {rel:.2e}, "
          f"low sweeps {rep.low_sweeps}, FP64 delta evals {rep.fp64_delta_evals}, deltas {rep.delta_fro}")
    assert rep.fp64_delta_evals >= 1 and rep.low_sweeps >= 2
    assert rep.delta_fro[-1] <= target
    assert resid <= 10 * target
    assert abs(resid_gpu - resid) <= 1e-3 * resid + 1e-13
    measured = {("chain", 1): 7.0e-5, ("chain", 2): 5.5e-4, ("cluster", 1): 7.2e-4, ("cluster", 2): 5.5e-3}
    assert rel <= 3 * measured[(kind, prec)]


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_refine_bs32(ctx, prec):
    """The mixed schedule at bs 32: TF32/BF16 sweeps on the narrow-tile
    tensor-core kernel (full products: the symmetric completion is built for
    bs 64), then delta with FP64-pipe products; the oracle's FP64 residual of
    the returned factor reaches the target."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(4096, 32, seed=0)
    tau, target = 1e-13, 1e-10
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), tau, target,
                                    ifac.opts(prec=prec, max_iter=80, delta_prec=0))
    a = Z.download()
    resid = oracle.resid(S, oracle.Mat(a.n, 32, a.row_ptr, a.col_idx, a.val))
    print(f"bs 32 prec={prec}: resid {resid:.2e}, low sweeps {rep.low_sweeps}, FP64 delta evals {rep.fp64_delta_evals}")
    assert rep.low_sweeps >= 2 and rep.fp64_delta_evals >= 1 and rep.tc_launches > 0
    assert resid <= 10 * target


@pytest.mark.parametrize("bs", [32, 128])
def test_mixed_refine_split_delta_block_sizes(ctx, bs):
    """The mixed schedule with split FP64-accurate delta at bs 32 and 128
    (TF32 sweeps on the narrow-tile kernel, delta on the narrow split kernel):
    the oracle's FP64 residual of the returned factor reaches the target."""
    from paper_1901_07993_gb300 import ifac
    S = synth.chain_overlap(4096, bs, seed=0)
    tau, target = 1e-13, 1e-10
    Z, rep = ifac.inv_factor_refine(ctx, ifac.upload(ctx, S), tau, target,
                                    ifac.opts(prec=1, max_iter=80, delta_prec=3))
    a = Z.download()
    resid = oracle.resid(S, oracle.Mat(a.n, bs, a.row_ptr, a.col_idx, a.val))
    print(f"bs {bs}: resid {resid:.2e}, low sweeps {rep.low_sweeps}, split delta evals {rep.fp64_delta_evals}")
    assert rep.split_launches > 0 and rep.tc_launches > 0
    assert resid <= 10 * target


def _same_factor(a, b):
    return (np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
            and np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64)))


@pytest.mark.parametrize("case", ["chain-tf32-narrow", "chain-bf16-narrow", "cluster-tf32-supertile",
                                  "chain-tf32-bs32", "batch-tf32"])
def test_fp32_intermediates_are_bitwise_neutral(ctx, case):
    """The low-precision products' results are FP32 accumulators, so keeping
    X, Z^T X, delta^2 and M in FP32 (ifac_set_fp32_intermediates, the default)
    must give bitwise the factors and delta norms of keeping them in FP64:
    narrow-tile and super-tile kernels, bs 64 and 32, single and batched."""
    from paper_1901_07993_gb300 import ifac
    prec = 2 if "bf16" in case else 1
    bs = 32 if "bs32" in case else 64
    if case.startswith("batch"):
        Ss = [synth.chain_overlap(1500, bs, seed=5), synth.cluster_overlap(700, bs, seed=2),
              synth.chain_overlap(2600, bs, seed=3)]
    elif case.startswith("cluster"):
        Ss = [synth.cluster_overlap(1024, bs, seed=0)]
    else:
        Ss = [synth.chain_overlap(4096, bs, seed=0)]
    dS = [ifac.upload(ctx, S) for S in Ss]
    if "supertile" in case:
        ifac.set_schedule(ctx, 0, -1)
    out = {}
    try:
        for on in (True, False):
            ctx.set_fp32_intermediates(on)
            if case.startswith("batch"):
                Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=prec))
            else:
                Z, rep = ifac.inv_factor_refine(ctx, dS[0], 1e-13, 1e-10, ifac.opts(prec=prec, max_iter=80))
                Zs, reps = [Z], [rep]
            out[on] = ([Z.download() for Z in Zs], [list(r.delta_fro) for r in reps], [r.sweeps for r in reps])
    finally:
        ctx.set_fp32_intermediates(True)
        ifac.set_schedule(ctx, -1, -1)
    (z1, d1, s1), (z0, d0, s0) = out[True], out[False]
    assert s1 == s0 and d1 == d0
    for a, b in zip(z1, z0):
        assert _same_factor(a, b)
