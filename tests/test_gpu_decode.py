"""GPU decode (mfa_decode_blocks, FP32) against the FP64 oracle on the same seeded inputs."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL_FP32, gm_blocks_fitted, oracle_decode_set, rel_errors
from oracle import bspline, decode

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


def _decode(mfa, ctx, bs, flags=0, **kw):
    blk = mfa.DeviceBlocks(bs)
    width = 1 if flags & mfa.DECODE_VALUE_ONLY else 4
    cache = torch.full((blk.nslots * blk.slot_voxels * width,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, blk.nslots, flags=flags, **kw)
    assert ctx.device_status() == 0
    return cache.view(blk.nslots, blk.slot_voxels, width).cpu().numpy()


def _slot_grid(cache, bs, b):
    nx, ny, nz = bs.nsamp[b]
    return cache[bs.slot[b], : nx * ny * nz].reshape(nz, ny, nx, -1)


def test_basis_tables_match_oracle(mfa, ctx):
    bs = synth.random_block_set(12, 101, ncp_choices=(2, 3, 4, 6, 9, 12, 20), nsamp_choices=(2, 5, 13, 32, 64),
                                nonuniform=True)
    blk = mfa.DeviceBlocks(bs)
    for b in range(len(bs)):
        span, basis = mfa.basis_tables(ctx, blk.desc[72 * b:72 * (b + 1)], blk.knots)
        span, basis = span.cpu().numpy(), basis.cpu().numpy()
        for a, t in enumerate(bs.block_knots(b)):
            p, n = bs.degree[b, a], bs.nsamp[b, a]
            u = bspline.sample_params(n)
            s = bspline.find_span(t, p, u)
            assert np.array_equal(span[a, :n], s)  # integer decision: bit-exact
            N, dN = bspline.basis(t, p, u), bspline.basis_deriv(t, p, u)
            for i in range(n):
                cols = np.arange(s[i] - p, s[i] + 1)
                assert np.max(np.abs(basis[a, i, 0, :p + 1] - N[i, cols])) < 2e-6
                scale = max(1.0, np.abs(dN).max())
                assert np.max(np.abs(basis[a, i, 1, :p + 1] - dN[i, cols])) < 2e-6 * scale
    assert ctx.device_status() == 0


@pytest.mark.parametrize("seed,nonuniform", [(201, False), (202, True), (203, True)])
def test_mixed_ragged_batch(mfa, ctx, seed, nonuniform):
    bs = synth.random_block_set(24, seed, ncp_choices=(2, 3, 4, 6, 8, 12, 16), degree_choices=(1, 2, 3),
                                nsamp_choices=(2, 3, 5, 13, 32, 33, 64), nonuniform=nonuniform)
    cache = _decode(mfa, ctx, bs)
    want = oracle_decode_set(bs)
    for b in range(len(bs)):
        ve, ge = rel_errors(_slot_grid(cache, bs, b), want[b])
        assert ve <= TOL_FP32 and max(ge) <= TOL_FP32, (b, ve, ge)


def test_value_only(mfa, ctx):
    bs = synth.random_block_set(10, 204, nsamp_choices=(5, 13, 32))
    cache = _decode(mfa, ctx, bs, flags=mfa.DECODE_VALUE_ONLY)
    want = oracle_decode_set(bs)
    for b in range(len(bs)):
        f = _slot_grid(cache, bs, b)[..., 0]
        w = want[b][..., 0]
        assert np.abs(f - w).max() / max(w.max() - w.min(), 1e-30) <= TOL_FP32


def test_single_block_16cp_on_64cubed(mfa, ctx):
    """One degree-2 block, 16^3 clamped uniform control points = Gaussian mixture at the Greville points,
    decoded on a 64^3 grid; compared voxel by voxel."""
    p, C, n = 2, 16, 64
    t = synth.clamped_uniform_knots(C, p)
    xi = synth.greville(t, p)
    Z, Y, X = np.meshgrid(xi, xi, xi, indexing="ij")
    P = synth.gm_params_field_at(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), synth.BASE_SEED + 1)
    bs = synth.make_block_set([(C, C, C)], [(p, p, p)], [(n, n, n)], [P.reshape(C, C, C)])
    cache = _decode(mfa, ctx, bs)
    want = oracle_decode_set(bs)[0]
    ve, ge = rel_errors(_slot_grid(cache, bs, 0), want)
    assert ve <= TOL_FP32 and max(ge) <= TOL_FP32, (ve, ge)


def test_gm_128cubed_c12_degree2(mfa, ctx):
    """The 512^3 Gaussian-mixture recipe reduced to 128^3 (64 blocks of 32^3, C = 12, degree 2, oracle least-squares control points)."""
    bs, _ = gm_blocks_fitted(128, 32, 12, 2, synth.BASE_SEED + 2)
    cache = _decode(mfa, ctx, bs)
    want = oracle_decode_set(bs)
    got = np.stack([_slot_grid(cache, bs, b) for b in range(len(bs))])
    ve, ge = rel_errors(got, np.stack(want))
    assert ve <= TOL_FP32 and max(ge) <= TOL_FP32, (ve, ge)


def test_gm_512cubed_4096_blocks_sampled(mfa, ctx):
    """The full 512^3 batch (4096 blocks of 32^3, C = 12, degree 2) decoded in one launch; 96 blocks x 400 voxels checked."""
    bs, _ = gm_blocks_fitted(512, 32, 12, 2, synth.BASE_SEED + 2, device="cuda")
    blk = mfa.DeviceBlocks(bs)
    cache = torch.empty(blk.nslots * blk.slot_voxels * 4, device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, blk.nslots)
    assert ctx.device_status() == 0
    cache = cache.view(blk.nslots, blk.slot_voxels, 4)
    g = synth.rng(7)
    got, want = [], []
    for b in g.choice(len(bs), 96, replace=False):
        kji = g.integers(0, 32, size=(400, 3))
        lin = torch.as_tensor((kji[:, 0] * 32 + kji[:, 1]) * 32 + kji[:, 2], device="cuda")
        got.append(cache[bs.slot[b]][lin].cpu().numpy())
        want.append(decode.decode_voxels(bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b], kji))
    ve, ge = rel_errors(np.concatenate(got), np.concatenate(want))
    assert ve <= TOL_FP32 and max(ge) <= TOL_FP32, (ve, ge)


def test_max_sizes(mfa, ctx):
    """Largest supported block: degree 3, 32 control points, 64 samples per axis."""
    g = synth.rng(205)
    p, C, n = 3, 32, 64
    P = g.uniform(-1, 1, (C, C, C))
    knots = [tuple(synth.random_clamped_knots(C, p, g) for _ in range(3))]
    bs = synth.make_block_set([(C, C, C)], [(p, p, p)], [(n, n, n)], [P], knots_list=knots)
    cache = _decode(mfa, ctx, bs)
    ve, ge = rel_errors(_slot_grid(cache, bs, 0), oracle_decode_set(bs)[0])
    assert ve <= TOL_FP32 and max(ge) <= TOL_FP32, (ve, ge)


def test_list_with_device_count_and_list_slots(mfa, ctx):
    bs = synth.random_block_set(16, 206, nsamp_choices=(8, 13))
    blk = mfa.DeviceBlocks(bs)
    order = np.array([5, 3, 11, 0, 7, 9], dtype=np.int32)
    lst = torch.as_tensor(order, device="cuda")
    count = torch.tensor([4], dtype=torch.int32, device="cuda")
    cache = torch.full((len(order) * blk.slot_voxels * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, len(order), list_=lst, count=count,
                      flags=mfa.DECODE_LIST_SLOTS)
    assert ctx.device_status() == 0
    c = cache.view(len(order), blk.slot_voxels, 4).cpu().numpy()
    for m, b in enumerate(order):
        nx, ny, nz = bs.nsamp[b]
        grid = c[m, : nx * ny * nz].reshape(nz, ny, nx, 4)
        if m < 4:
            ve, ge = rel_errors(grid, oracle_decode_set(bs, [b])[0])
            assert ve <= TOL_FP32 and max(ge) <= TOL_FP32
        else:
            assert np.all(np.isnan(grid))  # beyond the device count: untouched


def test_empty_batch_is_a_no_op(mfa, ctx):
    bs = synth.random_block_set(2, 207)
    blk = mfa.DeviceBlocks(bs)
    cache = torch.zeros(4 * blk.slot_voxels * 2, device="cuda")
    lst = torch.zeros(0, dtype=torch.int32, device="cuda")
    n0 = ctx.launch_count()
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 2, list_=lst)
    assert ctx.launch_count() == n0 and ctx.device_status() == 0
    count = torch.tensor([0], dtype=torch.int32, device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 2, list_=torch.zeros(4, dtype=torch.int32, device="cuda"),
                      count=count)
    assert ctx.device_status() == 0 and float(cache.abs().sum()) == 0.0


def test_device_side_checks_skip_bad_blocks(mfa, ctx):
    bs = synth.random_block_set(6, 208, ncp_choices=(4, 6), nsamp_choices=(8,))
    bs.knots = bs.knots.copy()
    # block 1: decreasing knots on x; block 2: slot out of range; block 4: list entry out of range
    t0 = bs.knot_off[1, 0]
    bad_knots = bs.knots.copy()
    kn = list(bs.block_knots(1)[0])
    bad_knots = np.concatenate([bad_knots, np.array(kn[::-1], dtype=np.float32)])
    bs.knot_off[1, 0] = len(bs.knots)
    bs.knots = bad_knots
    bs.slot[2] = 999
    blk = mfa.DeviceBlocks(bs)
    lst = torch.tensor([0, 1, 2, 3, 77, 5], dtype=torch.int32, device="cuda")
    cache = torch.full((6 * blk.slot_voxels * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 6, list_=lst)
    st = ctx.device_status()
    assert st & mfa.DEV_BAD_KNOTS and st & mfa.DEV_BAD_RANGE and st & mfa.DEV_BAD_LIST
    c = cache.view(6, blk.slot_voxels, 4).cpu().numpy()
    assert np.all(np.isnan(c[1])) and np.all(np.isfinite(c[0, :512])) and np.all(np.isfinite(c[5, :512]))
    assert ctx.device_status() == 0  # cleared


def test_bounds_violation_flags_bad_desc(mfa, ctx):
    bs = synth.random_block_set(3, 209, ncp_choices=(6,), nsamp_choices=(8,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    cache = torch.zeros(3 * blk.slot_voxels * 4, device="cuda")
    mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 3, bounds=mfa.Bounds(2, 5, 8))
    assert ctx.device_status() & mfa.DEV_BAD_DESC


def test_host_argument_checks(mfa, ctx):
    bs = synth.random_block_set(2, 210)
    blk = mfa.DeviceBlocks(bs)
    cache = torch.zeros(2 * blk.slot_voxels * 4 + 1, device="cuda")
    with pytest.raises(mfa.MfaError) as e:
        mfa.decode_blocks(ctx, blk, cache[1:], blk.slot_voxels, 2)  # misaligned cache
    assert e.value.code == mfa.ERR_INVALID_ARG
    with pytest.raises(mfa.MfaError) as e:
        mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 2, bounds=mfa.Bounds(4, 8, 8))
    assert e.value.code == mfa.ERR_INVALID_ARG
    with pytest.raises(mfa.MfaError) as e:
        mfa.decode_blocks(ctx, blk, cache, blk.slot_voxels, 2, flags=0x80)
    assert e.value.code == mfa.ERR_INVALID_ARG
    assert ctx.device_status() == 0
