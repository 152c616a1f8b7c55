"""GPU ray caster (mfa_raycast) against the oracle's Algorithm 4 on the same FP32 cache."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted, oracle_decode_set
from oracle import raycast as ocast

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


@pytest.fixture(scope="module")
def volume():
    """64^3 nodes = 4^3 bricks of 16^3, fitted with C = 8, degree 2; cache = oracle decode rounded to FP32."""
    bs, _ = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 12)
    cache = np.stack(oracle_decode_set(bs)).astype(np.float32)  # (64, 16, 16, 16, 4)
    return cache, 16


def _run(mfa, ctx, cache, table, n, view, tf):
    dev_cache = torch.from_numpy(cache.reshape(-1)).cuda()
    dev_table = torch.from_numpy(table.astype(np.int32)).cuda()
    dev_tf = torch.from_numpy(tf).cuda()
    img = torch.full((view["height"], view["width"], 4), float("nan"), device="cuda")
    mfa.raycast(ctx, dev_cache, n ** 3, cache.shape[0], dev_table, n, view, dev_tf, img)
    assert ctx.device_status() == 0
    return img.cpu().numpy()


def _tables(nb):
    ident = np.arange(nb ** 3, dtype=np.int32).reshape(nb, nb, nb)
    g = synth.rng(3)
    perm = g.permutation(nb ** 3).astype(np.int32)
    holes = ident.copy()
    holes[g.random(holes.shape) < 0.3] = -1
    return ident, perm, holes


@pytest.mark.parametrize("which", [0, 1, 2])
def test_raycast_no_early_termination(mfa, ctx, volume, which):
    cache, n = volume
    ident, perm, holes = _tables(4)
    table = [ident, perm, holes][which]
    if which == 1:  # permuted slots: the cache holds brick b at slot perm[b]
        c2 = np.empty_like(cache)
        c2[perm.reshape(-1)] = cache
        cache = c2
        table = perm.reshape(4, 4, 4)
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=64, height=48, opacity_max=1.0)
    got = _run(mfa, ctx, cache, table, n, view, tf)
    want = ocast.raycast(cache, table, n, view, tf)
    assert np.max(np.abs(got - want)) <= 1e-4


def test_raycast_early_termination_bound(mfa, ctx, volume):
    cache, n = volume
    ident, _, _ = _tables(4)
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    tf[:, 3] = np.clip(tf[:, 3] * 6, 0, 1)  # dense enough that most rays terminate early
    view = synth.default_view(width=64, height=64, opacity_max=0.99)
    got = _run(mfa, ctx, cache, ident, n, view, tf)
    want = ocast.raycast(cache, ident, n, view, tf)
    d = np.max(np.abs(got - want), axis=-1)
    assert (want[..., 3] > 0.99).mean() > 0.2
    assert d.max() <= 1e-2
    assert (d <= 1e-4).mean() >= 0.999


def test_raycast_constant_field_closed_form(mfa, ctx):
    n, B = 8, 2
    cache = np.zeros((B ** 3, n, n, n, 4), np.float32)
    cache[..., 0] = 0.5
    table = np.arange(B ** 3, dtype=np.int32).reshape(B, B, B)
    alpha = np.float32(0.05)
    tf = np.tile(np.array([0.2, 0.4, 0.8, alpha], np.float32), (16, 1))
    view = synth.default_view(width=5, height=5, eye=(0.0, 0.0, 3.0), opacity_max=1.0)
    got = _run(mfa, ctx, cache, table, n, view, tf)
    _, _, _, K, _ = ocast.ray_setup(view, (B * n,) * 3)
    assert K[2, 2] == B * n - 1
    A = 1 - (1 - np.float64(alpha)) ** K[2, 2]
    assert abs(got[2, 2, 3] - A) < 2e-6


def test_raycast_argument_checks(mfa, ctx, volume):
    cache, n = volume
    ident, _, _ = _tables(4)
    tf = synth.transfer_function(1)
    view = synth.default_view(width=8, height=8, vmin=1.0, vmax=1.0)
    with pytest.raises(mfa.MfaError):
        _run(mfa, ctx, cache, ident, n, view, tf)


def _fitted_volume(N, n, seed):
    bs, _ = gm_blocks_fitted(N, n, 8, 2, seed)
    return np.stack(oracle_decode_set(bs)).astype(np.float32)


def test_raycast_non_power_of_two_bricks(mfa, ctx):
    """Bricks of 12^3 (per-pixel tile kernel) against the oracle, with absent bricks."""
    n, nb = 12, 4
    cache = _fitted_volume(nb * n, n, synth.BASE_SEED + 13)
    _, _, holes = _tables(nb)
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=40, height=36, opacity_max=1.0)
    ctx.ray_samples(reset=True)
    got = _run(mfa, ctx, cache, holes, n, view, tf)
    marched = ctx.ray_samples(reset=True)
    want = ocast.raycast(cache, holes, n, view, tf)
    _, _, _, K, _ = ocast.ray_setup(view, (nb * n,) * 3)
    assert marched == int(np.asarray(K).sum())
    assert np.max(np.abs(got - want)) <= 1e-4


@pytest.mark.parametrize("wh", [(61, 37), (8, 4), (1, 1), (130, 3)])
def test_raycast_queue_ragged_image_and_sample_count(mfa, ctx, wh):
    """Bricks of 32^3 (persistent queue kernel), image sizes that are not multiples of the 8x4 warp tile.
    Without early termination every pixel marches exactly the K samples of its FP32 set-up, so the
    device's marched-sample counter equals the oracle's sum of K, and every pixel is written once."""
    n = 32
    cache = _fitted_volume(64, n, synth.BASE_SEED + 14)
    ident, _, _ = _tables(2)
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=wh[0], height=wh[1], opacity_max=1.0)
    ctx.ray_samples(reset=True)
    got = _run(mfa, ctx, cache, ident, n, view, tf)
    marched = ctx.ray_samples(reset=True)
    want = ocast.raycast(cache, ident, n, view, tf)
    _, _, _, K, _ = ocast.ray_setup(view, (2 * n,) * 3)
    assert not np.isnan(got).any()
    assert marched == int(np.asarray(K).sum())
    assert np.max(np.abs(got - want)) <= 1e-4


def test_raycast_half_voxel_steps_and_value_window(mfa, ctx, volume):
    """step_voxels = 1/2 (opacity correction 1 - (1 - a)^(1/2) per sample) and a value window narrower than
    the field's range (values outside it clamp to the end entries)."""
    cache, n = volume
    ident, _, holes = _tables(4)
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=48, height=40, opacity_max=1.0, step_voxels=0.5, vmin=0.2, vmax=0.8)
    for table in (ident, holes):
        got = _run(mfa, ctx, cache, table, n, view, tf)
        want = ocast.raycast(cache, table, n, view, tf)
        assert np.max(np.abs(got - want)) <= 1e-4


@pytest.mark.parametrize("N,n,holes", [(64, 16, False), (64, 16, True), (64, 32, False)])
def test_raycast_direct_model_queries_match_oracle(mfa, ctx, N, n, holes):
    """mfa_raycast_direct (per-sample queries of the fitted micro-models) against the oracle's direct renderer,
    early termination off; every pixel marches its K samples. Also reports how far the cache renderer's
    trilinear interpolation of the decoded nodes is from the direct queries (the cache discretisation)."""
    bs, _ = gm_blocks_fitted(N, n, 8, 2, synth.BASE_SEED + 18)
    B = N // n
    table = np.arange(B ** 3, dtype=np.int32).reshape(B, B, B)
    if holes:
        table[synth.rng(19).random(table.shape) < 0.3] = -1
    tf = synth.transfer_function(synth.BASE_SEED + 2)
    view = synth.default_view(width=40, height=32, opacity_max=1.0)
    blk = mfa.DeviceBlocks(bs)
    img = torch.full((view["height"], view["width"], 4), float("nan"), device="cuda")
    ctx.ray_samples(reset=True)
    mfa.raycast_direct(ctx, blk, torch.from_numpy(table).cuda(), n, view, torch.from_numpy(tf).cuda(), img)
    marched = ctx.ray_samples(reset=True)
    assert ctx.device_status() == 0
    got = img.cpu().numpy()
    want = ocast.raycast_direct(lambda k: (bs.block_cps(k), bs.block_knots(k), tuple(bs.degree[k])), table, n,
                                view, tf)
    _, _, _, K, _ = ocast.ray_setup(view, (N, N, N))
    assert marched == int(np.asarray(K).sum())
    assert np.max(np.abs(got - want)) <= 1e-4
    cache = np.stack(oracle_decode_set(bs)).astype(np.float32)
    via_cache = ocast.raycast(cache, table, n, view, tf)
    print(f"N={N} n={n} holes={holes}: max |direct - cache| = {np.max(np.abs(want - via_cache)):.2e}")


def _touched_sectors_host(view, B, n, stride, apron):
    """Distinct 32-byte cache sectors the eight corner loads of every sample read, replaying the FP32 sample
    positions the kernel forms (g = (fma(t_s, d, eye) + 1) * half + k * dg, one FMA per axis) with the
    oracle's FP32 ray set-up. Identity brick table, early termination off."""
    N = B * n
    d, t0, dt, K, eye = ocast.ray_setup(view, (N, N, N))
    f32 = np.float32
    half = f32((N - 1) / 2.0)

    def fma(a, b, c):  # FP32 fused multiply-add: exact product and sum in FP64, one rounding (ties aside)
        return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32)

    ts = fma(f32(0.5), dt, t0)
    gb = [((fma(ts, d[..., a], eye[a]) + f32(1.0)) * half).astype(f32) for a in range(3)]
    dg = [((dt * d[..., a]).astype(f32) * half).astype(f32) for a in range(3)]
    A = (n + 1 + 1) // 2 * 2 if apron else n
    P = n + 1 if apron else n
    secs = set()
    for y, x in zip(*np.nonzero(K > 0)):
        k = np.arange(K[y, x], dtype=np.float64)
        g = [np.clip(fma(k.astype(f32), dg[a][y, x], gb[a][y, x]), 0, N - 1) for a in range(3)]
        i = [np.minimum(g[a].astype(np.int64), N - 2) for a in range(3)]
        slot = ((i[2] // n) * B + i[1] // n) * B + i[0] // n
        for e in range(8):
            dx, dy, dz = e & 1, (e >> 1) & 1, e >> 2
            lx, ly, lz = i[0] % n + dx, i[1] % n + dy, i[2] % n + dz
            if not apron:  # a corner beyond the brick reads the neighbour's first plane
                sl = (((i[2] + dz) // n) * B + (i[1] + dy) // n) * B + (i[0] + dx) // n
                vox = sl * stride + (((i[2] + dz) % n) * n + (i[1] + dy) % n) * n + (i[0] + dx) % n
            else:
                vox = slot * stride + (lz * P + ly) * A + lx
            secs.update((vox >> 1).tolist())
    return len(secs)


@pytest.mark.parametrize("apron", [False, True])
def test_raycast_sector_count(mfa, ctx, apron):
    """MFA_RAYCAST_COUNT_SECTORS renders the same image bit for bit and counts the distinct 32-byte cache
    sectors of the corner loads: equal to a host replay of the kernel's sample cells (to 0.5 %: a sample
    exactly on a cell boundary may round the other way), and below the cache's sector count."""
    n, B = 16, 2
    cache = _fitted_volume(B * n, n, synth.BASE_SEED + 15)
    table = torch.arange(B ** 3, dtype=torch.int32, device="cuda").view(B, B, B)
    tf = torch.from_numpy(synth.transfer_function(synth.BASE_SEED + 2)).cuda()
    view = synth.default_view(width=48, height=40, opacity_max=1.0)
    S = mfa.apron_voxels(n) if apron else n ** 3
    dev = torch.zeros(B ** 3, S, 4, device="cuda")
    if apron:
        A = mfa.apron_pitch(n)
        dev[:, : (n + 1) * (n + 1) * A].view(B ** 3, n + 1, n + 1, A, 4)[:, :n, :n, :n] = torch.from_numpy(cache).cuda()
        mfa.fill_aprons(ctx, dev, S, B ** 3, table, n)
    else:
        dev.copy_(torch.from_numpy(cache.reshape(B ** 3, S, 4)))
    img = [torch.full((40, 48, 4), float("nan"), device="cuda") for _ in range(2)]
    ctx.stats(reset=True)
    mfa.raycast(ctx, dev, S, B ** 3, table, n, view, tf, img[0], apron=apron)
    mfa.raycast(ctx, dev, S, B ** 3, table, n, view, tf, img[1], apron=apron, count_sectors=True)
    st = ctx.stats(reset=True)
    assert ctx.device_status() == 0
    assert torch.equal(img[0], img[1])
    want = _touched_sectors_host(view, B, n, S, apron)
    assert abs(st[mfa.STAT_RAY_SECTORS] - want) <= 0.005 * want, (st, want)
    assert st[mfa.STAT_RAY_SECTORS] <= B ** 3 * S // 2
