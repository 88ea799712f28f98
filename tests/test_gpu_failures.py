"""Failure paths of the C ABI on the GPU, none of which faults the device:

- an allocator that fails on its k-th call: the call returns IFAC_ERR_OOM,
  every buffer the library took from that allocator is returned by the time
  the call returns (nothing leaks), and the context stays usable;
- max_iter reached: IFAC_ERR_NO_CONVERGENCE (FP64 and mixed schedules),
  as in the oracle, which stops with the same reason at the same sweep;
- an expired bounded wait inside the tensor-core pipeline
  (ifac_selftest_wait_timeout: a launch whose copy and MMA stages do no work,
  so the epilogue's wait runs out): IFAC_ERR_TIMEOUT, after which the same
  context still computes bit-identical products.
"""
import numpy as np
import pytest

import oracle
from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    assert torch.cuda.is_available()
    libbuild.build()
    return ifac


class CountingAllocator:
    """torch's caching allocator behind the library's allocator interface;
    returns NULL on call number fail_at (1-based), and tracks live buffers."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        import torch
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=int(stream))
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        import torch
        assert ptr in self.live, "free of a pointer the allocator did not hand out"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def _refine(ifac, ctx, S, prec):
    dS = ifac.upload(ctx, S)
    return ifac.inv_factor_refine(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=prec, max_iter=60))


@pytest.mark.parametrize("prec", [0, 1])
def test_oom_on_kth_allocation_leaks_nothing(lib, prec):
    import torch
    ifac = lib
    S = synth.chain_overlap(4096, 64, seed=0)
    # a full run through the counting allocator: the number of allocations
    ok = CountingAllocator()
    ctx = ifac.Context(allocator=(ok.alloc, ok.free))
    Z, rep = _refine(ifac, ctx, S, prec)
    n_calls = ok.calls
    held = len(ok.live)  # the returned Z's four arrays
    assert held == 4
    Z_ok = Z.download()
    del Z
    torch.cuda.synchronize()
    assert not ok.live and n_calls > 20
    for k in sorted({2, 5, n_calls // 7, n_calls // 3, n_calls // 2, n_calls - 1, n_calls}):
        fa = CountingAllocator(fail_at=k)
        c = ifac.Context(allocator=(fa.alloc, fa.free))
        dS = ifac.upload(c, S) if k > 4 else None  # the upload itself takes the first 4 allocations
        owned = set(fa.live)  # the caller's S (nothing when the upload is the call that fails)
        with pytest.raises(ifac.IfacError) as ei:
            if dS is None:
                dS = ifac.upload(c, S)
            ifac.inv_factor_refine(c, dS, 1e-12, 1e-10, ifac.opts(prec=prec, max_iter=60))
        code = ei.value.code
        del ei  # its traceback holds the caller's S
        assert code == ifac.ERR_OOM, k
        torch.cuda.synchronize()
        # everything the failed call allocated has been returned
        assert set(fa.live) == owned, (k, len(fa.live), len(owned))
        del dS
        assert not fa.live, (k, len(fa.live))
        # the context is still usable: the same factorization, the same result
        fa.fail_at = None
        Z2, _ = _refine(ifac, c, S, prec)
        z2 = Z2.download()
        assert np.array_equal(z2.col_idx, Z_ok.col_idx) and np.array_equal(z2.val, Z_ok.val), k
        del Z2
        c.close()
        torch.cuda.synchronize()
        assert not fa.live


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_max_iter_gives_no_convergence(lib, prec):
    ifac = lib
    ctx = ifac.Context()
    S = synth.chain_overlap(2048, 64, seed=1)
    dS = ifac.upload(ctx, S)
    with pytest.raises(ifac.IfacError) as ei:
        ifac.inv_factor_refine(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=prec, max_iter=1))
    assert ei.value.code == ifac.ERR_NO_CONVERGENCE
    # the oracle stops for the same reason after the same single sweep
    _, rep = oracle.irsi(S, tau=1e-12, target=1e-10, max_iter=1)
    assert rep.stop_reason == ifac.STOP_MAXITER and rep.sweeps == 1
    # and the context still factorizes
    Z, rep = ifac.inv_factor_refine(ctx, dS, 1e-12, 1e-10, ifac.opts(prec=prec, max_iter=60))
    assert rep.delta_fro[-1] <= 1e-10


def test_wait_timeout_reports_and_context_survives(lib):
    ifac = lib
    ctx = ifac.Context()
    A = synth.random_bsr(6, 64, 0.5, seed=3)
    dA = ifac.upload(ctx, A)
    before = ifac.bsr_gemm_trunc(ctx, dA, False, dA, True, 1.0, 0.0, ifac.TF32).download()
    assert ifac.selftest_wait_timeout(ctx, 1 << 20) == ifac.ERR_TIMEOUT
    assert ifac.selftest_wait_timeout(ctx, 0) == ifac.ERR_INVALID
    after = ifac.bsr_gemm_trunc(ctx, dA, False, dA, True, 1.0, 0.0, ifac.TF32).download()
    assert np.array_equal(before.col_idx, after.col_idx) and np.array_equal(before.val, after.val)
    # a second expiry in a row behaves the same
    assert ifac.selftest_wait_timeout(ctx, 1 << 18) == ifac.ERR_TIMEOUT
    again = ifac.bsr_gemm_trunc(ctx, dA, False, dA, True, 1.0, 0.0, ifac.TF32).download()
    assert np.array_equal(before.val, again.val)
