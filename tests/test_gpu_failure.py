"""Failure detection on the GPU without a fault: the bounded mbarrier wait gives up on a barrier that nothing
arrives on, reports MFA_DEV_TIMEOUT in the context's status word, and leaves the context usable."""

import pytest
import torch

import synth
from gpu_util import TOL_FP32, oracle_decode_set, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfa():
    from paper_2409_00184_b300 import mfa as m
    return m


@pytest.fixture(scope="module")
def ctx(mfa):
    c = mfa.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("polls", [1, 1000])
def test_bounded_wait_times_out_and_context_stays_usable(mfa, ctx, polls):
    assert ctx.device_status() == 0
    ctx.selftest_wait_timeout(polls)
    assert ctx.device_status() == mfa.DEV_TIMEOUT  # the read synchronises and clears the word
    assert ctx.device_status() == 0
    # the same context (and its tensor-core and TMA kernels) still produce correct results
    bs = synth.random_block_set(6, 801, ncp_choices=(4, 8, 12), nsamp_choices=(32,), degree_choices=(2, 3))
    blk = mfa.DeviceBlocks(bs)
    for prec, tol in ((mfa.PREC_FP32, TOL_FP32), (mfa.PREC_SPLIT_BF16, 1e-4)):
        cache = torch.full((blk.nslots * blk.slot_voxels * 4,), float("nan"), device="cuda")
        mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, blk.nslots, precision=prec)
        assert ctx.device_status() == 0
        got = cache.view(blk.nslots, 32, 32, 32, 4).cpu().numpy()
        want = oracle_decode_set(bs)
        for b in range(len(bs)):
            ve, ge = rel_errors(got[bs.slot[b]], want[b])
            assert ve <= tol and max(ge) <= tol, (prec, b, ve, ge)


def test_selftest_argument_checks(mfa, ctx):
    for polls in (0, -1, (1 << 20) + 1):
        with pytest.raises(mfa.MfaError):
            ctx.selftest_wait_timeout(polls)
    assert ctx.device_status() == 0


def test_host_device_copies_round_trip():
    """mfa_copy_to_device / mfa_copy_to_host move pinned host bytes to the device and back unchanged, and
    refuse null pointers and negative sizes."""
    import ctypes
    import torch
    from paper_2409_00184_b300 import mfa
    torch.cuda.set_device(0)
    h = torch.arange(1 << 20, dtype=torch.float32).pin_memory()
    d = torch.empty_like(h, device="cuda")
    back = torch.zeros_like(h).pin_memory()
    s = torch.cuda.Stream()
    mfa.copy_to_device(d, h, stream=s)
    mfa.copy_to_host(back, d, stream=s)
    s.synchronize()
    assert torch.equal(back, h)
    assert mfa.lib.mfa_copy_to_device(None, ctypes.c_void_p(h.data_ptr()), 4, None) == mfa.ERR_INVALID_ARG
    assert mfa.lib.mfa_copy_to_host(ctypes.c_void_p(back.data_ptr()), ctypes.c_void_p(d.data_ptr()), -1,
                                    None) == mfa.ERR_INVALID_ARG


def test_binding_refuses_tensors_of_another_element_type(mfa, ctx):
    """The binding checks each tensor's element type before a call: a byte tensor as the cache would pass an
    element-count check yet be a quarter of the bytes the decode writes. Nothing is launched."""
    bs = synth.random_block_set(2, 811, ncp_choices=(4,), nsamp_choices=(8,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    n0 = ctx.launch_count()
    V = blk.slot_voxels
    with pytest.raises(ValueError):
        mfa.decode_blocks(ctx, blk, torch.zeros(2 * V * 4, dtype=torch.uint8, device="cuda"), V, 2)
    with pytest.raises(ValueError):
        mfa.decode_blocks(ctx, blk, torch.zeros(2 * V * 4, device="cuda"), V, 2,
                          list_=torch.zeros(2, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        mfa.adjoint_blocks(ctx, blk, torch.zeros(2 * V, dtype=torch.float64, device="cuda"), V, 2,
                           torch.zeros(blk.cps_len, device="cuda"))
    table = torch.zeros(1, 1, 2, dtype=torch.int32, device="cuda")
    view = synth.default_view(width=8, height=8)
    tf = torch.from_numpy(synth.transfer_function(1)).cuda()
    cache = torch.zeros(2 * V * 4, device="cuda")
    with pytest.raises(ValueError):  # a transfer function must be (n, 4)
        mfa.raycast(ctx, cache, V, 2, table, 8, view, tf.view(-1), torch.zeros(8, 8, 4, device="cuda"))
    with pytest.raises(ValueError):
        mfa.raycast(ctx, cache, V, 2, table.long(), 8, view, tf, torch.zeros(8, 8, 4, device="cuda"))
    with pytest.raises(ValueError):
        mfa.raycast(ctx, cache, V, 2, table, 8, view, tf, torch.zeros(8, 8, 4, dtype=torch.float64, device="cuda"))
    assert ctx.launch_count() == n0 and ctx.device_status() == 0
