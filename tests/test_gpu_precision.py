"""Tensor-core decode (tcgen05) in BF16, FP16 and split-BF16 against the FP64 oracle.

Tolerances (relative to the value range / the largest gradient component, per precision): split-BF16
1e-4, plain BF16 1e-2, FP16 1e-2. Errors of each variant are printed for the record.
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted, oracle_decode_set, rel_errors
from oracle import decode as odec

pytestmark = pytest.mark.gpu

TOL = {"split": 1e-4, "bf16": 1e-2, "fp16": 1e-2}


@pytest.fixture(scope="module")
def mfa():
    from paper_2409_00184_b300 import mfa as m
    return m


@pytest.fixture(scope="module")
def ctx(mfa):
    c = mfa.Context(0)
    yield c
    c.close()


def _prec(mfa, name):
    return {"split": mfa.PREC_SPLIT_BF16, "bf16": mfa.PREC_BF16, "fp16": mfa.PREC_FP16}[name]


def _decode(mfa, ctx, bs, precision, **kw):
    blk = mfa.DeviceBlocks(bs)
    cache = torch.full((blk.nslots * blk.slot_voxels * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, blk.nslots, precision=precision, **kw)
    return cache.view(blk.nslots, blk.slot_voxels, 4).cpu().numpy()


@pytest.mark.parametrize("name", ["split", "bf16", "fp16"])
@pytest.mark.parametrize("degree", [2, 3])
def test_tensor_core_decode_fitted_blocks(mfa, ctx, name, degree):
    """64 fitted blocks of 32^3 (Gaussian mixture + noise, C = 12)."""
    bs, _ = gm_blocks_fitted(128, 32, 12, degree, synth.BASE_SEED + 4)
    got = _decode(mfa, ctx, bs, _prec(mfa, name))
    assert ctx.device_status() == 0
    want = np.stack(oracle_decode_set(bs))
    ve, ge = rel_errors(got.reshape(len(bs), 32, 32, 32, 4), want)
    print(f"{name} degree {degree}: value {ve:.2e}, gradient {max(ge):.2e}")
    assert ve <= TOL[name] and max(ge) <= TOL[name], (ve, ge)


@pytest.mark.parametrize("name", ["split", "bf16"])
def test_tensor_core_decode_mixed_shapes(mfa, ctx, name):
    """Anisotropic C in 2..16, degrees 1..3, non-uniform knots, all with 32 samples per axis (one sub-cube)."""
    bs = synth.random_block_set(20, 601, ncp_choices=(2, 3, 4, 7, 12, 16), degree_choices=(1, 2, 3),
                                nsamp_choices=(32,), nonuniform=True)
    got = _decode(mfa, ctx, bs, _prec(mfa, name))
    assert ctx.device_status() == 0
    want = oracle_decode_set(bs)
    for b in range(len(bs)):
        ve, ge = rel_errors(got[bs.slot[b]].reshape(32, 32, 32, 4), want[b])
        assert ve <= TOL[name] and max(ge) <= TOL[name], (b, ve, ge)


def test_tensor_core_list_slots_and_shape_checks(mfa, ctx):
    bs = synth.random_block_set(8, 602, ncp_choices=(6, 8), nsamp_choices=(32,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    order = torch.tensor([6, 1, 3], dtype=torch.int32, device="cuda")
    cnt = torch.tensor([2], dtype=torch.int32, device="cuda")
    cache = torch.full((3 * 32 ** 3 * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, 32 ** 3, 3, precision=mfa.PREC_SPLIT_BF16, list_=order, count=cnt,
                      flags=mfa.DECODE_LIST_SLOTS)
    assert ctx.device_status() == 0
    c = cache.view(3, 32 ** 3, 4).cpu().numpy()
    for m, b in enumerate([6, 1]):
        ve, ge = rel_errors(c[m].reshape(32, 32, 32, 4), oracle_decode_set(bs, [b])[0])
        assert ve <= 1e-4 and max(ge) <= 1e-4
    assert np.all(np.isnan(c[2]))
    # outside the tensor-core path: the cube layout (host refusal), and a sub-cube whose samples' bands cover
    # more than 16 control points (clustered knots: a per-block device flag, the other blocks decode)
    with pytest.raises(mfa.MfaError) as e:
        mfa.decode_blocks(ctx, blk, torch.zeros(3 * 32 ** 3 * 4, device="cuda"), 32 ** 3, 3,
                          precision=mfa.PREC_BF16, flags=mfa.DECODE_CUBES)
    assert e.value.code == mfa.ERR_UNSUPPORTED
    C, p = 24, 2
    uni = synth.clamped_uniform_knots(C, p)
    clustered = np.concatenate([np.zeros(p + 1), np.linspace(0.01, 0.3, C - p - 1), np.ones(p + 1)])
    gm = synth.rng(605)
    mixed = synth.make_block_set([(C, C, C)] * 3, [(p, p, p)] * 3, [(32, 32, 32)] * 3,
                                 [gm.uniform(-1, 1, size=(C, C, C)) for _ in range(3)],
                                 [(uni, uni, uni), (uni, clustered, uni), (uni, uni, uni)])
    mblk = mfa.DeviceBlocks(mixed)
    cache = torch.full((3 * mblk.slot_voxels * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, mblk, cache, mblk.slot_voxels, 3, precision=mfa.PREC_BF16)
    assert ctx.device_status() & mfa.DEV_BAD_DESC  # reading the status clears it
    c = cache.view(3, mblk.slot_voxels, 4).cpu().numpy()
    want = oracle_decode_set(mixed, [0, 2])
    for m, b in enumerate([0, 2]):
        ve, ge = rel_errors(c[mixed.slot[b]].reshape(32, 32, 32, 4), want[m])
        assert ve <= 1e-2 and max(ge) <= 1e-2
    # the flagged block's sub-cubes with y < 16 (the window of 22 control points) are not written
    assert np.all(np.isnan(c[mixed.slot[1]].reshape(32, 32, 32, 4)[:, :16]))


@pytest.mark.parametrize("name", ["split", "bf16", "fp16"])
def test_tensor_core_decode_empty_and_clamped_counts(mfa, ctx, name):
    """Empty inputs of the tensor-core decode: no blocks (the call returns before any launch), a device count of
    0 (the kernel runs and writes nothing), and a device count above the list's length (MFA_DEV_BAD_LIST, and
    the count is clamped to the list: every listed block is decoded, nothing else)."""
    import ctypes
    prec = _prec(mfa, name)
    bs = synth.random_block_set(4, 611, ncp_choices=(6, 12), nsamp_choices=(32,), degree_choices=(2, 3))
    blk = mfa.DeviceBlocks(bs)
    V = blk.slot_voxels
    cache = torch.full((4 * V * 4,), float("nan"), device="cuda")
    n0 = ctx.launch_count()
    rc = mfa.lib.mfa_decode_blocks(ctx.handle, ctypes.c_void_p(blk.desc.data_ptr()), 0, None, 0, None,
                                   ctypes.c_void_p(blk.knots.data_ptr()), blk.knots.numel(),
                                   ctypes.c_void_p(blk.cps.data_ptr()), blk.cps.numel(),
                                   ctypes.c_void_p(cache.data_ptr()), V, 4, ctypes.byref(blk.bounds), prec, 0,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mfa.OK and ctx.launch_count() == n0
    lst = torch.tensor([2, 0, 3, 1], dtype=torch.int32, device="cuda")
    mfa.decode_blocks(ctx, blk, cache, V, 4, precision=prec, list_=lst,
                      count=torch.tensor([0], dtype=torch.int32, device="cuda"), flags=mfa.DECODE_LIST_SLOTS)
    assert ctx.launch_count() > n0 and ctx.device_status() == 0
    assert torch.isnan(cache).all()
    lst3 = lst[:3].contiguous()
    mfa.decode_blocks(ctx, blk, cache, V, 4, precision=prec, list_=lst3,
                      count=torch.tensor([9], dtype=torch.int32, device="cuda"), flags=mfa.DECODE_LIST_SLOTS)
    assert ctx.device_status() == mfa.DEV_BAD_LIST
    c = cache.view(4, V, 4).cpu().numpy()
    want = oracle_decode_set(bs, [2, 0, 3])
    for m in range(3):
        ve, ge = rel_errors(c[m, : 32 ** 3].reshape(32, 32, 32, 4), want[m])
        assert ve <= TOL[name] and max(ge) <= TOL[name], (m, ve, ge)
    assert np.all(np.isnan(c[3]))


@pytest.mark.parametrize("name", ["split", "bf16", "fp16"])
def test_tensor_core_decode_any_sample_count(mfa, ctx, name):
    """Sample counts other than 32 (2 .. 64 per axis, anisotropic, non-uniform knots): a block of n samples is
    decoded as ceil(n/32)^3 sub-cubes whose rows past n are zero and never stored."""
    bs = synth.random_block_set(14, 606, ncp_choices=(2, 3, 5, 9, 16), degree_choices=(1, 2, 3),
                                nsamp_choices=(2, 7, 16, 31, 33, 48, 64), nonuniform=True)
    got = _decode(mfa, ctx, bs, _prec(mfa, name))
    assert ctx.device_status() == 0
    want = oracle_decode_set(bs)
    for b in range(len(bs)):
        nx, ny, nz = (int(v) for v in bs.nsamp[b])
        vox = nx * ny * nz
        ve, ge = rel_errors(got[bs.slot[b]][:vox].reshape(nz, ny, nx, 4), want[b])
        assert ve <= TOL[name] and max(ge) <= TOL[name], (b, bs.nsamp[b], ve, ge)
        assert np.all(np.isnan(got[bs.slot[b]][vox:]))  # nothing written past the block's voxels


@pytest.mark.parametrize("name", ["split", "bf16", "fp16"])
def test_tensor_core_decode_more_than_16_control_points(mfa, ctx, name):
    """C up to 24 per axis (uniform knots, n >= 32, degrees 1..3, mixed with C <= 16): axes with C > 16 are
    decoded in 16-sample sub-cubes, each over the window of at most 16 control points its bands cover."""
    bs = synth.random_block_set(12, 607, ncp_choices=(4, 12, 17, 20, 24), degree_choices=(1, 2, 3),
                                nsamp_choices=(32, 40, 64))
    got = _decode(mfa, ctx, bs, _prec(mfa, name))
    assert ctx.device_status() == 0
    want = oracle_decode_set(bs)
    assert int(np.max(bs.ncp)) > 16
    for b in range(len(bs)):
        nx, ny, nz = (int(v) for v in bs.nsamp[b])
        vox = nx * ny * nz
        ve, ge = rel_errors(got[bs.slot[b]][:vox].reshape(nz, ny, nx, 4), want[b])
        assert ve <= TOL[name] and max(ge) <= TOL[name], (b, bs.ncp[b], bs.nsamp[b], ve, ge)


def test_tensor_core_list_count_with_sub_cubes(mfa, ctx):
    """A device list and count with list slots, over blocks of several sub-cubes each (n = 48 and C up to 20:
    27 sub-cube positions per item): every listed block lands in its list slot, unlisted slots stay unwritten."""
    bs = synth.random_block_set(6, 609, ncp_choices=(5, 12, 20), degree_choices=(2, 3), nsamp_choices=(33, 48))
    blk = mfa.DeviceBlocks(bs)
    order = torch.tensor([4, 0, 5, 2], dtype=torch.int32, device="cuda")
    cnt = torch.tensor([3], dtype=torch.int32, device="cuda")
    V = blk.slot_voxels
    cache = torch.full((4 * V * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, V, 4, precision=mfa.PREC_SPLIT_BF16, list_=order, count=cnt,
                      flags=mfa.DECODE_LIST_SLOTS)
    assert ctx.device_status() == 0
    c = cache.view(4, V, 4).cpu().numpy()
    want = oracle_decode_set(bs, [4, 0, 5])
    for m, b in enumerate([4, 0, 5]):
        nx, ny, nz = (int(v) for v in bs.nsamp[b])
        ve, ge = rel_errors(c[m][:nx * ny * nz].reshape(nz, ny, nx, 4), want[m])
        assert ve <= TOL["split"] and max(ge) <= TOL["split"], (b, ve, ge)
    assert np.all(np.isnan(c[3]))


def test_tensor_core_decode_adaptive_ncp(mfa, ctx):
    """Blocks of the adaptive-NCP batch's classes ({4, 6, 8, 12, 16, 20, 24} per axis, degree 2, 32^3
    samples) in one split-BF16 launch against the oracle."""
    g = synth.rng(608)
    classes = (4, 6, 8, 12, 16, 20, 24)
    ncp = [tuple(int(v) for v in g.choice(classes, 3)) for _ in range(24)]
    ncp[0] = (24, 24, 24)
    bs = synth.make_block_set(ncp, [(2, 2, 2)] * len(ncp), [(32, 32, 32)] * len(ncp),
                              [g.uniform(0, 1, size=c[::-1]) for c in ncp])
    got = _decode(mfa, ctx, bs, mfa.PREC_SPLIT_BF16)
    assert ctx.device_status() == 0
    want = np.stack(oracle_decode_set(bs))
    ve, ge = rel_errors(got.reshape(len(bs), 32, 32, 32, 4), want)
    print(f"adaptive NCP split-BF16: value {ve:.2e}, gradient {max(ge):.2e}")
    assert ve <= TOL["split"] and max(ge) <= TOL["split"], (ve, ge)


@pytest.mark.parametrize("apron", [False, True])
def test_tensor_core_value_only(mfa, ctx, apron):
    """MFA_DECODE_VALUE_ONLY on the tensor cores writes f alone (one float per voxel), equal bit for bit to the
    f of the full decode, in the row and in the apron layout."""
    bs = synth.random_block_set(10, 610, ncp_choices=(4, 12, 20), degree_choices=(2, 3), nsamp_choices=(16, 32, 40))
    blk = mfa.DeviceBlocks(bs)
    S = max(mfa.apron_voxels(int(v)) for v in bs.nsamp.max(axis=1)) if apron else blk.slot_voxels
    base = mfa.DECODE_APRON if apron else 0
    full = torch.full((blk.nslots * S * 4,), float("nan"), device="cuda")
    val = torch.full((blk.nslots * S,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, full, S, blk.nslots, precision=mfa.PREC_SPLIT_BF16, flags=base)
    mfa.decode_blocks(ctx, blk, val, S, blk.nslots, precision=mfa.PREC_SPLIT_BF16,
                      flags=base | mfa.DECODE_VALUE_ONLY)
    assert ctx.device_status() == 0
    f4 = full.view(blk.nslots, S, 4)[..., 0].cpu().numpy()
    v = val.view(blk.nslots, S).cpu().numpy()
    assert np.array_equal(np.isnan(f4), np.isnan(v))
    assert np.array_equal(f4[~np.isnan(f4)], v[~np.isnan(v)])


def test_tensor_core_decode_single_block_16cp_on_64cubed(mfa, ctx):
    """On the tensor cores: one block of 16^3 control points (degree 2, Gaussian-mixture samples)
    decoded on a 64^3 grid in split-BF16 (eight 32^3 sub-cubes), every voxel against the oracle."""
    C, p, n = 16, 2, 64
    g = synth.rng(synth.BASE_SEED + 1)
    cps = g.uniform(0.0, 1.0, size=(C, C, C))
    t = synth.clamped_uniform_knots(C, p)
    bs = synth.make_block_set([(C, C, C)], [(p, p, p)], [(n, n, n)], [cps], [(t, t, t)])
    got = _decode(mfa, ctx, bs, mfa.PREC_SPLIT_BF16)
    assert ctx.device_status() == 0
    ve, ge = rel_errors(got[0].reshape(n, n, n, 4), oracle_decode_set(bs)[0])
    print(f"one 16^3-control-point block, split-BF16: value {ve:.2e}, gradient {max(ge):.2e}")
    assert ve <= TOL["split"] and max(ge) <= TOL["split"], (ve, ge)


def test_degree3_512cubed_4096_blocks_sampled(mfa, ctx):
    """The degree-3 512^3 batch (4096 blocks, 12^3 control points) at degree 3, every precision, sampled
    voxels against the oracle; prints max and RMS error of value and gradient per variant."""
    bs, _ = gm_blocks_fitted(512, 32, 12, 3, synth.BASE_SEED + 4, device="cuda")
    blk = mfa.DeviceBlocks(bs)
    cache = torch.empty(blk.nslots * blk.slot_voxels * 4, device="cuda")
    g = synth.rng(44)
    picks = [(b, g.integers(0, 32, size=(300, 3))) for b in g.choice(len(bs), 64, replace=False)]
    want = np.concatenate([odec.decode_voxels(bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b], kji)
                           for b, kji in picks])
    for name, prec in [("fp32", mfa.PREC_FP32), ("split", mfa.PREC_SPLIT_BF16), ("bf16", mfa.PREC_BF16),
                       ("fp16", mfa.PREC_FP16)]:
        mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, blk.nslots, precision=prec)
        assert ctx.device_status() == 0
        c = cache.view(blk.nslots, blk.slot_voxels, 4)
        got = np.concatenate([c[b][torch.as_tensor((k[:, 0] * 32 + k[:, 1]) * 32 + k[:, 2], device="cuda")]
                             .cpu().numpy() for b, k in picks])
        ve, ge = rel_errors(got, want)
        print(f"degree-3 512^3 {name}: value {ve:.2e} gradient {max(ge):.2e}")
        assert ve <= TOL.get(name, 1e-5) and max(ge) <= TOL.get(name, 1e-5), (name, ve, ge)


@pytest.mark.parametrize("name", ["fp32", "split", "bf16"])
def test_decode_with_repeated_interior_knots(mfa, ctx, name):
    """Knot vectors with repeated interior knots (multiplicity up to p): the FP32 decode and the tensor-core
    decode against the oracle, with sample counts from 13 to 64."""
    from gpu_util import TOL_FP32, repeated_knot_set
    bs = repeated_knot_set(10, 351, nsamp_choices=(13, 32, 64))
    prec = mfa.PREC_FP32 if name == "fp32" else _prec(mfa, name)
    got = _decode(mfa, ctx, bs, prec)
    assert ctx.device_status() == 0
    want = oracle_decode_set(bs)
    tol = TOL_FP32 if name == "fp32" else TOL[name]
    for b in range(len(bs)):
        nx, ny, nz = bs.nsamp[b]
        ve, ge = rel_errors(got[bs.slot[b], : nx * ny * nz].reshape(nz, ny, nx, 4), want[b])
        assert ve <= tol and max(ge) <= tol, (b, ve, ge)
