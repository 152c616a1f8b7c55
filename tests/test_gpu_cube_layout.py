"""The cube layout of the decoded cache (MFA_DECODE_CUBES, mfa_raycast_ex with MFA_RAYCAST_CUBES,
MFA_FRAME_CUBES): the same voxels as the [z][y][x] layout, permuted, and the same images bit for bit.
The row layout itself is checked against the FP64 oracle elsewhere; here the permutation is written out
from its definition (cube index 8*((z/2*ny/2 + y/2)*nx/2 + x/2) + 4*(z%2) + 2*(y%2) + x%2)."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted, oracle_decode_set

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


def cube_order(nx, ny, nz):
    """perm[v_cube] = v_row for the voxels of one nx x ny x nz brick."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = (((z // 2) * (ny // 2) + y // 2) * (nx // 2) + x // 2) * 8 + (z % 2) * 4 + (y % 2) * 2 + (x % 2)
    perm = np.empty(nx * ny * nz, dtype=np.int64)
    perm[cube.reshape(-1)] = np.arange(nx * ny * nz)
    return perm


def to_cubes(cache, n):
    """(slots, n, n, n, 4) row-layout bricks -> the same bricks in the cube layout, (slots, n^3, 4)."""
    flat = cache.reshape(cache.shape[0], n ** 3, -1)
    return np.ascontiguousarray(flat[:, cube_order(n, n, n)])


def test_cube_order_is_a_permutation_with_cubes_in_lines():
    perm = cube_order(4, 6, 8)
    assert sorted(perm.tolist()) == list(range(4 * 6 * 8))
    # every aligned group of 8 cube-layout entries is one 2x2x2 cube of row-layout voxels
    for g in range(0, perm.size, 8):
        z, r = np.divmod(perm[g:g + 8], 24)
        y, x = np.divmod(r, 4)
        assert np.ptp(x) == 1 and np.ptp(y) == 1 and np.ptp(z) == 1 and x.min() % 2 == 0


@pytest.mark.parametrize("value_only", [False, True])
def test_decode_cubes_permutes_the_row_layout(mfa, ctx, value_only):
    bs = synth.random_block_set(10, 611, ncp_choices=(4, 6, 8, 12), nsamp_choices=(8, 12, 32), degree_choices=(1, 2, 3))
    blk = mfa.DeviceBlocks(bs)
    width = 1 if value_only else 4
    S = blk.slot_voxels
    row = torch.full((blk.nslots * S * width,), float("nan"), device="cuda")
    cub = torch.full_like(row, float("nan"))
    base = mfa.DECODE_VALUE_ONLY if value_only else 0
    mfa.decode_blocks(ctx, blk, row, S, blk.nslots, flags=base)
    mfa.decode_blocks(ctx, blk, cub, S, blk.nslots, flags=base | mfa.DECODE_CUBES)
    assert ctx.device_status() == 0
    row = row.view(blk.nslots, S, width).cpu().numpy()
    cub = cub.view(blk.nslots, S, width).cpu().numpy()
    for b in range(len(bs)):
        nx, ny, nz = (int(v) for v in bs.nsamp[b])
        s, vox = bs.slot[b], nx * ny * nz
        assert np.array_equal(cub[s, :vox], row[s, cube_order(nx, ny, nz)]), b


def test_decode_compare_cubes(mfa, ctx):
    bs, D = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 21)
    blk = mfa.DeviceBlocks(bs)
    S = blk.slot_voxels
    data = torch.from_numpy(np.ascontiguousarray(D.reshape(len(bs), -1), dtype=np.float32)).cuda().view(-1)
    outs = []
    for flags in (0, mfa.DECODE_CUBES):
        cache = torch.full((blk.nslots * S * 4,), float("nan"), device="cuda")
        res = torch.full_like(data, float("nan"))
        rm = torch.zeros(len(bs), dtype=torch.float64, device="cuda")
        mfa.decode_compare_blocks(ctx, blk, cache, S, blk.nslots, data, S, residual=res, rmse=rm, flags=flags)
        assert ctx.device_status() == 0
        outs.append((cache.view(blk.nslots, S, 4).cpu().numpy(), res.cpu().numpy(), rm.cpu().numpy()))
    (c0, r0, m0), (c1, r1, m1) = outs
    assert np.array_equal(r0, r1) and np.array_equal(m0, m1)
    assert np.array_equal(c1, c0[:, cube_order(16, 16, 16)])


def test_decode_cubes_rejects_odd_sizes_and_other_precisions(mfa, ctx):
    bs = synth.random_block_set(3, 612, ncp_choices=(4,), nsamp_choices=(9,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    S = blk.slot_voxels
    cache = torch.full((blk.nslots * S * 4,), 7.0, device="cuda")
    mfa.decode_blocks(ctx, blk, cache, S, blk.nslots, flags=mfa.DECODE_CUBES)
    assert ctx.device_status() == mfa.DEV_BAD_DESC
    assert bool((cache == 7.0).all())  # skipped blocks leave their slots untouched
    with pytest.raises(mfa.MfaError):
        mfa.decode_blocks(ctx, blk, cache, S, blk.nslots, precision=mfa.PREC_BF16, flags=mfa.DECODE_CUBES)
    assert ctx.device_status() == 0


@pytest.fixture(scope="module")
def volume():
    """64^3 nodes = 4^3 bricks of 16^3 (FP32 oracle decode): the ray caster's queue kernel (n = 2^4)."""
    bs, _ = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 12)
    return np.stack(oracle_decode_set(bs)).astype(np.float32), 16


def _render(mfa, ctx, cache_flat, nslots, table, n, view, tf, cubes):
    dev_cache = torch.from_numpy(np.ascontiguousarray(cache_flat).reshape(-1)).cuda()
    img = torch.full((view["height"], view["width"], 4), float("nan"), device="cuda")
    mfa.raycast(ctx, dev_cache, n ** 3, nslots, torch.from_numpy(table.astype(np.int32)).cuda(), n, view,
                torch.from_numpy(tf).cuda(), img, cubes=cubes)
    assert ctx.device_status() == 0
    return img.cpu().numpy()


@pytest.mark.parametrize("holes", [False, True])
def test_raycast_cubes_matches_rows_bitwise(mfa, ctx, volume, holes):
    cache, n = volume
    table = np.arange(64, dtype=np.int32).reshape(4, 4, 4)
    if holes:
        table[synth.rng(5).random(table.shape) < 0.3] = -1
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=75, height=53)  # ragged warp tiles; cells across bricks
    rows = _render(mfa, ctx, cache, 64, table, n, view, tf, False)
    cubes = _render(mfa, ctx, to_cubes(cache, n), 64, table, n, view, tf, True)
    assert np.isfinite(rows).all() and rows[..., 3].max() > 0.1
    assert np.array_equal(rows, cubes)


def test_raycast_cubes_any_even_brick(mfa, ctx):
    """Bricks of 6^3 (not a power of two: the per-pixel kernel) from random values."""
    g = synth.rng(14)
    n, nb = 6, 3
    cache = g.uniform(0, 1, (nb ** 3, n, n, n, 4)).astype(np.float32)
    table = g.permutation(nb ** 3).astype(np.int32).reshape(nb, nb, nb)
    tf = synth.transfer_function(synth.BASE_SEED + 3)
    view = synth.default_view(width=40, height=36, vmin=0.0, vmax=1.0)
    rows = _render(mfa, ctx, cache, nb ** 3, table, n, view, tf, False)
    cubes = _render(mfa, ctx, to_cubes(cache, n), nb ** 3, table, n, view, tf, True)
    assert np.array_equal(rows, cubes)
    with pytest.raises(mfa.MfaError):  # the cube layout needs an even brick size
        _render(mfa, ctx, cache[:, :5, :5, :5].copy(), nb ** 3, table, 5, view, tf, True)


def test_frame_graph_cubes(mfa, ctx):
    bs, _ = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 12)
    blk = mfa.DeviceBlocks(bs)
    S, B = blk.slot_voxels, len(bs)
    ids = torch.from_numpy(synth.rng(8).permutation(B)[:40].astype(np.int32)).cuda()
    tf = torch.from_numpy(synth.transfer_function(synth.BASE_SEED + 2)).cuda()
    view = synth.default_view(width=64, height=64)
    images = []
    for cubes in (False, True):
        lst = torch.zeros(B, dtype=torch.int32, device="cuda")
        cnt = torch.tensor([40], dtype=torch.int32, device="cuda")
        lst[:40] = ids
        cache = torch.zeros(B * S * 4, device="cuda")
        table = torch.empty(B, dtype=torch.int32, device="cuda")
        img = torch.zeros(64, 64, 4, device="cuda")
        fg = mfa.FrameGraph(ctx, blk, lst, cnt, cache, S, sort=True, table=table, brick_dims=(4, 4, 4), brick_n=16,
                            view=view, tf=tf, image=img, cubes=cubes)
        fg.launch()
        assert ctx.device_status() == 0
        images.append(img.cpu().numpy())
        fg.close()
    assert images[0][..., 3].max() > 0.05
    assert np.array_equal(images[0], images[1])
