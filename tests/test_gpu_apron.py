"""The apron layout of the decoded cache (MFA_DECODE_APRON, mfa_fill_aprons, MFA_RAYCAST_APRON,
MFA_FRAME_APRON): bricks of n^3 voxels stored in rows of A = n + 1 rounded up to even voxels, planes of
n + 1 rows and n + 1 planes, with the planes x = n, y = n, z = n copied from the neighbouring bricks and
the columns n < x < A zero. The interior is the row-layout decode in that addressing, the aprons follow
their definition (written out here in numpy), and the ray caster's images equal the row layout's bit for
bit."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted, oracle_decode_set

pytestmark = pytest.mark.gpu


def pitch(n):
    return -(-(n + 1) // 2) * 2


def apron_voxels(n):
    """Voxels of one apron slot: n + 1 planes of n + 1 rows of pitch(n)."""
    return pitch(n) * (n + 1) ** 2


@pytest.fixture(scope="module")
def mfa():
    from paper_2409_00184_b300 import mfa as m
    return m


@pytest.fixture(scope="module")
def ctx(mfa):
    c = mfa.Context(0)
    yield c
    c.close()


def with_aprons(cache, table, n):
    """Row-layout bricks (slots, n, n, n, 4) -> (slots, apron_voxels(n), 4) with interiors copied and the
    apron of every brick of `table` ((Bz, By, Bx) slots, -1 absent) taken from its neighbours; zeros
    elsewhere (the padding columns x > n included)."""
    S, p = cache.shape[0], n + 1
    out = np.zeros((S, p, p, pitch(n), 4), np.float32)
    out[:, :n, :n, :n] = cache
    Bz, By, Bx = table.shape
    for bz in range(Bz):
        for by in range(By):
            for bx in range(Bx):
                s = table[bz, by, bx]
                if s < 0:
                    continue
                for z in range(p):
                    for y in range(p):
                        for x in range(p):
                            if x < n and y < n and z < n:
                                continue
                            sx, sy, sz = bx + (x == n), by + (y == n), bz + (z == n)
                            v = 0.0
                            if sx < Bx and sy < By and sz < Bz and table[sz, sy, sx] >= 0:
                                v = cache[table[sz, sy, sx], z % n, y % n, x % n]
                            out[s, z, y, x] = v
    return out.reshape(S, apron_voxels(n), 4)


def test_decode_apron_writes_the_interior_with_pitch(mfa, ctx):
    bs = synth.random_block_set(8, 811, ncp_choices=(4, 6, 8), nsamp_choices=(7, 12, 16), degree_choices=(1, 2, 3))
    blk = mfa.DeviceBlocks(bs)
    S = max(pitch(int(nx)) * (int(ny) + 1) * (int(nz) + 1) for nx, ny, nz in bs.nsamp)
    for vo in (False, True):
        w = 1 if vo else 4
        base = mfa.DECODE_VALUE_ONLY if vo else 0
        row = torch.full((blk.nslots * S * w,), float("nan"), device="cuda")
        apr = torch.full_like(row, float("nan"))
        mfa.decode_blocks(ctx, blk, row, S, blk.nslots, flags=base)
        mfa.decode_blocks(ctx, blk, apr, S, blk.nslots, flags=base | mfa.DECODE_APRON)
        assert ctx.device_status() == 0
        row = row.view(blk.nslots, S, w).cpu().numpy()
        apr = apr.view(blk.nslots, S, w).cpu().numpy()
        for b in range(len(bs)):
            nx, ny, nz = (int(v) for v in bs.nsamp[b])
            s = bs.slot[b]
            a = apr[s, : pitch(nx) * (ny + 1) * (nz + 1)].reshape(nz + 1, ny + 1, pitch(nx), w)
            assert np.array_equal(a[:nz, :ny, :nx], row[s, : nx * ny * nz].reshape(nz, ny, nx, w)), b
            assert np.isnan(a[nz]).all() and np.isnan(a[:, ny]).all() and np.isnan(a[:, :, nx:]).all()


def test_fill_aprons_follows_the_definition(mfa, ctx):
    g = synth.rng(31)
    n, dims = 6, (3, 2, 4)  # (Bx, By, Bz)
    nb = dims[0] * dims[1] * dims[2]
    cache = g.uniform(-1, 1, (nb, n, n, n, 4)).astype(np.float32)
    table = g.permutation(nb).astype(np.int32).reshape(dims[2], dims[1], dims[0])
    table[g.random(table.shape) < 0.25] = -1
    want = with_aprons(cache, table, n)
    p3 = apron_voxels(n)
    dev = torch.full((nb, p3, 4), float("nan"), device="cuda")
    dev.view(nb, n + 1, n + 1, pitch(n), 4)[:, :n, :n, :n] = torch.from_numpy(cache).cuda()
    mfa.fill_aprons(ctx, dev.view(-1), p3, nb, torch.from_numpy(table).cuda(), n)
    assert ctx.device_status() == 0
    got = dev.cpu().numpy()
    used = sorted(set(table[table >= 0].tolist()))
    assert np.array_equal(got[used], want[used])
    unused = [s for s in range(nb) if s not in used]  # slots of absent bricks are not touched
    assert all(np.isnan(got[s].reshape(n + 1, n + 1, pitch(n), 4)[n]).all() for s in unused)


@pytest.fixture(scope="module")
def volume():
    """64^3 nodes = 4^3 bricks of 16^3 (FP32 oracle decode)."""
    bs, _ = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 12)
    return np.stack(oracle_decode_set(bs)).astype(np.float32), 16


def _render(mfa, ctx, cache_flat, stride, nslots, table, n, view, tf, apron):
    dev_cache = torch.from_numpy(np.ascontiguousarray(cache_flat).reshape(-1)).cuda()
    img = torch.full((view["height"], view["width"], 4), float("nan"), device="cuda")
    mfa.raycast(ctx, dev_cache, stride, nslots, torch.from_numpy(table.astype(np.int32)).cuda(), n, view,
                torch.from_numpy(tf).cuda(), img, apron=apron)
    assert ctx.device_status() == 0
    return img.cpu().numpy()


@pytest.mark.parametrize("which", ["ident", "perm", "holes"])
def test_raycast_apron_matches_rows_bitwise(mfa, ctx, volume, which):
    cache, n = volume
    g = synth.rng(6)
    table = np.arange(64, dtype=np.int32).reshape(4, 4, 4)
    if which == "perm":
        perm = g.permutation(64).astype(np.int32)
        c2 = np.empty_like(cache)
        c2[perm] = cache
        cache, table = c2, perm.reshape(4, 4, 4)
    if which == "holes":
        table[g.random(table.shape) < 0.3] = -1
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=75, height=53)
    rows = _render(mfa, ctx, cache, n ** 3, 64, table, n, view, tf, False)
    apr = _render(mfa, ctx, with_aprons(cache, table, n), apron_voxels(n), 64, table, n, view, tf, True)
    assert np.isfinite(rows).all() and rows[..., 3].max() > 0.1
    assert np.array_equal(rows, apr)


@pytest.mark.parametrize("holes", [False, True])
@pytest.mark.parametrize("n", [5, 6])
def test_raycast_apron_any_brick_size(mfa, ctx, n, holes):
    """Bricks of 5^3 (pitch 6, no padding column) and 6^3 (pitch 8): not powers of two, the per-pixel
    kernel; with absent bricks, cells whose own brick is absent read their present neighbours' corners."""
    g = synth.rng(15 + n)
    nb = 3
    cache = g.uniform(0, 1, (nb ** 3, n, n, n, 4)).astype(np.float32)
    table = g.permutation(nb ** 3).astype(np.int32).reshape(nb, nb, nb)
    if holes:
        table[g.random(table.shape) < 0.3] = -1
    tf = synth.transfer_function(synth.BASE_SEED + 3)
    view = synth.default_view(width=40, height=36)
    rows = _render(mfa, ctx, cache, n ** 3, nb ** 3, table, n, view, tf, False)
    apr = _render(mfa, ctx, with_aprons(cache, table, n), apron_voxels(n), nb ** 3, table, n, view, tf, True)
    assert np.array_equal(rows, apr)


def test_decode_compare_apron(mfa, ctx):
    bs, D = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 21)
    blk = mfa.DeviceBlocks(bs)
    V, P3 = 16 ** 3, apron_voxels(16)
    data = torch.from_numpy(np.ascontiguousarray(D.reshape(len(bs), -1), dtype=np.float32)).cuda().view(-1)
    outs = []
    for flags, stride in ((0, V), (mfa.DECODE_APRON, P3)):
        cache = torch.full((blk.nslots * stride * 4,), float("nan"), device="cuda")
        res = torch.full_like(data, float("nan"))
        rm = torch.zeros(len(bs), dtype=torch.float64, device="cuda")
        mfa.decode_compare_blocks(ctx, blk, cache, stride, blk.nslots, data, V, residual=res, rmse=rm, flags=flags)
        assert ctx.device_status() == 0
        outs.append((cache.view(blk.nslots, stride, 4).cpu().numpy(), res.cpu().numpy(), rm.cpu().numpy()))
    (c0, r0, m0), (c1, r1, m1) = outs
    assert np.array_equal(r0, r1) and np.array_equal(m0, m1)
    assert np.array_equal(c1.reshape(-1, 17, 17, pitch(16), 4)[:, :16, :16, :16], c0.reshape(-1, 16, 16, 16, 4))


def test_frame_graph_apron(mfa, ctx):
    bs, _ = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 12)
    blk = mfa.DeviceBlocks(bs)
    B = len(bs)
    ids = torch.from_numpy(synth.rng(9).permutation(B)[:40].astype(np.int32)).cuda()
    tf = torch.from_numpy(synth.transfer_function(synth.BASE_SEED + 2)).cuda()
    view = synth.default_view(width=64, height=64)
    images = []
    for apron in (False, True):
        S = apron_voxels(16) if apron else 16 ** 3
        lst = torch.zeros(B, dtype=torch.int32, device="cuda")
        cnt = torch.tensor([40], dtype=torch.int32, device="cuda")
        lst[:40] = ids
        cache = torch.zeros(B * S * 4, device="cuda")
        table = torch.empty(B, dtype=torch.int32, device="cuda")
        img = torch.zeros(64, 64, 4, device="cuda")
        fg = mfa.FrameGraph(ctx, blk, lst, cnt, cache, S, sort=True, table=table, brick_dims=(4, 4, 4), brick_n=16,
                            view=view, tf=tf, image=img, apron=apron)
        fg.launch()
        assert ctx.device_status() == 0
        images.append(img.cpu().numpy())
        fg.close()
    assert images[0][..., 3].max() > 0.05
    assert np.array_equal(images[0], images[1])


def test_apron_argument_checks(mfa, ctx):
    bs = synth.random_block_set(2, 812, ncp_choices=(4,), nsamp_choices=(8,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    cache = torch.full((2 * apron_voxels(8) * 4,), 3.0, device="cuda")
    with pytest.raises(mfa.MfaError):  # cubes and apron together
        mfa.decode_blocks(ctx, blk, cache, apron_voxels(8), 2, flags=mfa.DECODE_APRON | mfa.DECODE_CUBES)
    with pytest.raises(mfa.MfaError):  # tensor-core precisions write the row or the apron layout, not cubes
        mfa.decode_blocks(ctx, blk, cache, apron_voxels(8), 2, precision=mfa.PREC_BF16, flags=mfa.DECODE_CUBES)
    for prec in (mfa.PREC_FP32, mfa.PREC_BF16):  # slots one voxel short
        mfa.decode_blocks(ctx, blk, cache, apron_voxels(8) - 1, 2, precision=prec, flags=mfa.DECODE_APRON)
        assert ctx.device_status() == mfa.DEV_BAD_RANGE
    assert bool((cache == 3.0).all())
    table = torch.zeros(1, 1, 1, dtype=torch.int32, device="cuda")
    with pytest.raises(mfa.MfaError):
        mfa.fill_aprons(ctx, cache, apron_voxels(8) - 1, 2, table, 8)
    img = torch.zeros(8, 8, 4, device="cuda")
    tf = torch.from_numpy(synth.transfer_function(1)).cuda()
    with pytest.raises(mfa.MfaError):
        mfa.raycast(ctx, cache, apron_voxels(8) - 1, 2, table, 8, synth.default_view(width=8, height=8), tf, img,
                    apron=True)
    # a frame graph that fills and ray-casts with aprons needs the apron slot too (checked at creation)
    lst = torch.arange(2, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([2], dtype=torch.int32, device="cuda")
    tab = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(mfa.MfaError):
        mfa.FrameGraph(ctx, blk, lst, cnt, cache, 8 ** 3, sort=False, table=tab, brick_dims=(2, 1, 1), brick_n=8,
                       view=synth.default_view(width=8, height=8), tf=tf, image=img, apron=True)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("prec", ["split", "bf16"])
@pytest.mark.parametrize("N,n,C", [(128, 32, 12), (64, 16, 8)])
def test_tensor_core_decode_apron(mfa, ctx, prec, N, n, C):
    """The tensor-core decode in the apron layout: the interior equals its row-layout decode bit for bit,
    the apron planes are left to mfa_fill_aprons, and after the fill the apron ray cast equals the row
    layout's bit for bit."""
    precision = {"split": mfa.PREC_SPLIT_BF16, "bf16": mfa.PREC_BF16}[prec]
    bs, _ = gm_blocks_fitted(N, n, C, 2, synth.BASE_SEED + 13)
    blk = mfa.DeviceBlocks(bs)
    B, P3 = len(bs), apron_voxels(n)
    row = torch.full((B * n ** 3 * 4,), float("nan"), device="cuda")
    apr = torch.full((B * P3 * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, row, n ** 3, B, precision=precision)
    mfa.decode_blocks(ctx, blk, apr, P3, B, precision=precision, flags=mfa.DECODE_APRON)
    assert ctx.device_status() == 0
    r = row.view(B, n, n, n, 4).cpu().numpy()
    a = apr.view(B, n + 1, n + 1, pitch(n), 4).cpu().numpy()
    assert np.array_equal(a[:, :n, :n, :n], r)
    assert np.isnan(a[:, n]).all() and np.isnan(a[:, :, n]).all() and np.isnan(a[:, :, :, n:]).all()
    nb = N // n
    table = np.arange(B, dtype=np.int32).reshape(nb, nb, nb)
    mfa.fill_aprons(ctx, apr, P3, B, torch.from_numpy(table).cuda(), n)
    assert ctx.device_status() == 0
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=64, height=48)
    img_rows = _render(mfa, ctx, r, n ** 3, B, table, n, view, tf, False)
    img_apr = _render(mfa, ctx, apr.cpu().numpy(), P3, B, table, n, view, tf, True)
    assert img_rows[..., 3].max() > 0.1
    assert np.array_equal(img_rows, img_apr)
