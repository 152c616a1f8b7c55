"""The allocation-free encode entry point against the plan-based one, through the C ABI.

mfa_encode_blocks_noalloc serves callers that cannot allocate device memory (their device memory
belongs to another runtime's pool, or their frame loop must not stall on cudaMalloc/cudaFree): it
keeps its scratch in a fixed device array inside the library. Two calls in a row, on batches with
different shapes, must each give the plan-based encode's control points and RMSE; the second call
also shows that the shared scratch does not carry state from the first.
"""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _batch(seed):
    g = synth.rng(seed)
    bs = synth.random_block_set(24, seed, nsamp_choices=(8, 13, 32), ncp_choices=(3, 4, 6, 8, 12))
    stride = int(np.max(np.prod(bs.nsamp.astype(np.int64), axis=1)))
    data = g.uniform(-1, 1, (len(bs), stride)).astype(np.float32)
    return bs, data, stride


def test_noalloc_encode_matches_plan_encode_twice():
    from paper_2409_00184_b300 import mfa
    torch.cuda.set_device(0)
    ctx = mfa.Context(0)
    for seed in (901, 902):
        bs, data, stride = _batch(seed)
        blk = mfa.DeviceBlocks(bs)
        D = torch.from_numpy(data.ravel()).cuda()
        plan = mfa.EncodePlan(ctx, blk)
        want = torch.full((blk.cps_len,), float("nan"), device="cuda")
        want_rmse = torch.full((len(bs),), float("nan"), dtype=torch.float64, device="cuda")
        mfa.encode_blocks(ctx, plan, D, stride, len(bs), want, want_rmse)
        assert ctx.device_status() == 0
        plan.close()
        got = torch.full((blk.cps_len,), float("nan"), device="cuda")
        got_rmse = torch.full((len(bs),), float("nan"), dtype=torch.float64, device="cuda")
        mfa.encode_blocks_noalloc(blk, D, stride, len(bs), got, got_rmse)
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - w).max() <= 1e-5 * max(1.0, np.abs(w).max())
        wr, gr = want_rmse.cpu().numpy(), got_rmse.cpu().numpy()
        assert np.abs(gr - wr).max() <= 1e-5 * (data.max() - data.min())
    ctx.close()


def test_noalloc_encode_without_rmse_takes_the_zfirst_fit():
    """Without an RMSE buffer, with at most 16 control points and 32 samples per axis, 16-byte-aligned data and
    a slot stride that is a multiple of 32, the fit runs on the z-first kernel, which reads the pseudo-inverses
    and basis tables from the fixed scratch: two calls in a row against the plan-based encode."""
    from paper_2409_00184_b300 import mfa
    torch.cuda.set_device(0)
    ctx = mfa.Context(0)
    for seed in (904, 905):
        bs = synth.random_block_set(40, seed, nsamp_choices=(16, 32), ncp_choices=(4, 6, 8, 12, 16))
        stride = 32 ** 3
        data = synth.rng(seed).uniform(-1, 1, (len(bs), stride)).astype(np.float32)
        blk = mfa.DeviceBlocks(bs)
        D = torch.from_numpy(data.ravel()).cuda()
        assert D.data_ptr() % 16 == 0
        plan = mfa.EncodePlan(ctx, blk)
        want = torch.full((blk.cps_len,), float("nan"), device="cuda")
        mfa.encode_blocks(ctx, plan, D, stride, len(bs), want)
        assert ctx.device_status() == 0
        plan.close()
        got = torch.full((blk.cps_len,), float("nan"), device="cuda")
        mfa.encode_blocks_noalloc(blk, D, stride, len(bs), got)
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - w).max() <= 1e-5 * max(1.0, np.abs(w).max())
    ctx.close()


def test_noalloc_encode_rejects_a_batch_beyond_its_scratch():
    from paper_2409_00184_b300 import mfa
    torch.cuda.set_device(0)
    # 80 blocks with their own random knots: 240 distinct 32x64 axis classes need 1.97 MB of
    # pseudo-inverses and 0.31 MB of basis tables, more than the 2 MiB scratch
    g = synth.rng(903)
    B, C, n, p = 80, 32, 64, 3
    knots = [tuple(synth.random_clamped_knots(C, p, g, 0.02) for _ in range(3)) for _ in range(B)]
    bs = synth.make_block_set([(C,) * 3] * B, [(p,) * 3] * B, [(n,) * 3] * B, [np.zeros((C, C, C))] * B,
                              knots_list=knots)
    blk = mfa.DeviceBlocks(bs)
    D = torch.zeros(B * n ** 3, device="cuda")
    out = torch.zeros(blk.cps_len, device="cuda")
    with pytest.raises(mfa.MfaError) as e:
        mfa.encode_blocks_noalloc(blk, D, n ** 3, B, out)
    assert e.value.code == mfa.ERR_CAPACITY
