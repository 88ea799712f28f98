"""The allocation-free leaf inverse Cholesky (leaf_invchol_batched_noalloc).

It exists for callers that cannot allocate device memory when they need the
leaf routine (hosts that own the whole device-memory budget, loops that
cannot pay an allocation's synchronisation with the device): it takes its
scratch from a fixed 32 MiB device array inside the library instead of the
context's allocator.

Called through the C ABI with ctypes, twice in a row per case (the shared
scratch keeps the previous call's contents), its output must match the
allocating entry point leaf_invchol_batched within the tolerance the other
leaf tests use, and the oracle's dense inverse Cholesky factor.  The
in-place form (S == Z) is run too, and a partial overlap of S and Z is
rejected.  Kept in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_1901_07993_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _spd_batch(count, nl, seed):
    mats = []
    for k in range(count):
        if nl % 32 == 0:
            mats.append(synth.cluster_overlap(nl, 32, seed=seed + k).to_dense()[:nl, :nl])
        else:
            mats.append(synth.chain_overlap(nl, 8, seed=seed + k).to_dense()[:nl, :nl])
    return np.array(mats)


@pytest.mark.parametrize("count,nl", [(4, 128), (3, 200), (2, 512)])
def test_noalloc_matches_allocating_leaf_routine(count, nl):
    import torch

    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac

    libbuild.build()
    lib = ifac.load()
    fn = lib.leaf_invchol_batched_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    ctx = ifac.Context()
    stream = torch.cuda.current_stream().cuda_stream

    S = torch.tensor(_spd_batch(count, nl, seed=11), device="cuda")
    Z_ref, info_ref, rc_ref = ifac.leaf_invchol_batched(ctx, S)
    assert rc_ref == 0
    Z_ref = Z_ref.cpu().numpy()

    import oracle
    Sh = S.cpu().numpy()
    Z_or = [oracle.invchol(Sh[k]) for k in range(count)]
    for k in range(count):
        err = np.linalg.norm(Z_ref[k] - Z_or[k]) / np.linalg.norm(Z_or[k])
        assert err <= TOL, ("allocating routine vs oracle", k, err)

    for call in range(2):
        Z = torch.full_like(S, float("nan"))
        info = torch.full((count,), -1, dtype=torch.int32, device="cuda")
        rc = fn(stream, count, nl, S.data_ptr(), Z.data_ptr(), info.data_ptr())
        assert rc == ifac.OK, (call, rc)
        torch.cuda.current_stream().synchronize()
        assert info.cpu().tolist() == [0] * count
        Zh = Z.cpu().numpy()
        for k in range(count):
            err = np.linalg.norm(Zh[k] - Z_ref[k]) / np.linalg.norm(Z_ref[k])
            assert err <= TOL, (call, k, err)
            err = np.linalg.norm(Zh[k] - Z_or[k]) / np.linalg.norm(Z_or[k])
            assert err <= TOL, ("vs oracle", call, k, err)

    # in place (S == Z): the factors overwrite the inputs
    for call in range(2):
        W = S.clone()
        info = torch.full((count,), -1, dtype=torch.int32, device="cuda")
        rc = fn(stream, count, nl, W.data_ptr(), W.data_ptr(), info.data_ptr())
        assert rc == ifac.OK, ("in place", call, rc)
        torch.cuda.current_stream().synchronize()
        assert info.cpu().tolist() == [0] * count
        Wh = W.cpu().numpy()
        for k in range(count):
            err = np.linalg.norm(Wh[k] - Z_ref[k]) / np.linalg.norm(Z_ref[k])
            assert err <= TOL, ("in place", call, k, err)


def test_noalloc_reports_not_spd_and_rejects_oversize():
    import torch

    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac

    libbuild.build()
    ctx = ifac.Context()
    stream = torch.cuda.current_stream().cuda_stream
    S = _spd_batch(2, 64, seed=3)
    S[1, 40, 40] = -1.0
    St = torch.tensor(S, device="cuda")
    _, info_ref, rc_ref = ifac.leaf_invchol_batched(ctx, St)
    assert rc_ref == ifac.ERR_NOT_SPD
    for _ in range(2):
        Z = torch.empty_like(St)
        info = torch.zeros(2, dtype=torch.int32, device="cuda")
        assert ifac.leaf_invchol_batched_noalloc(stream, St, Z, info) == ifac.OK
        torch.cuda.current_stream().synchronize()
        assert info.cpu().tolist() == info_ref.cpu().tolist() == [0, 41]
    # 200 leaves of 1000 rows need 200 * 32 * 1024 tile-inverse doubles alone,
    # more than the 4 Mi-double array: rejected before any copy or launch
    count, nl = 200, 1000
    np_ = (nl + 31) // 32 * 32
    assert count * (np_ // 32) * 1024 > 4 * 2 ** 20
    tiny = torch.zeros((1, 1, 1), dtype=torch.float64, device="cuda")
    rc = ifac.load().leaf_invchol_batched_noalloc(stream, count, nl, tiny.data_ptr(), tiny.data_ptr(),
                                                  tiny.data_ptr())
    assert rc == ifac.ERR_TOO_LARGE
    # S and Z overlapping without being equal: rejected before any copy
    buf = torch.tensor(np.concatenate([S, S]), device="cuda")
    before = buf.clone()
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    off = 64 * 64 * 8  # Z starts one matrix into S
    rc = ifac.load().leaf_invchol_batched_noalloc(stream, 2, 64, buf.data_ptr(), buf.data_ptr() + off,
                                                  info.data_ptr())
    assert rc == ifac.ERR_INVALID
    torch.cuda.current_stream().synchronize()
    assert torch.equal(buf, before)
