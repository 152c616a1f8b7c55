"""Out-of-core rendering (Algorithms 2-4) on the GPU: the cache's upload reproduces the stored models, and
frames rendered through the store, the LRU cache and prefetching equal frames rendered from models that
are resident on the device."""

import numpy as np
import pytest
import torch

import synth
from test_gpu_frames import flame_blockset
from test_model_store import isotropic_blocks

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


def test_upload_reproduces_the_stored_models(mfa, ctx, tmp_path):
    bs = isotropic_blocks(30, 1200)
    path = tmp_path / "m.mfa"
    mfa.store_write(path, bs)
    cache = mfa.ModelCache(path, capacity=10, pinned=True)
    ids = np.array([7, 3, 29, 0, 12], dtype=np.int32)
    cache.lookup(ids)
    batch = mfa.DeviceBatch(10, int(bs.ncp.max()), int(bs.degree.max()))
    cache.upload(ids, 16, batch)
    torch.cuda.synchronize()
    desc = batch.desc.cpu().numpy().view(mfa.DESC_DTYPE)[: len(ids)]
    knots, cps = batch.knots.cpu().numpy(), batch.cps.cpu().numpy()
    for i, b in enumerate(ids):
        d = desc[i]
        assert tuple(d["ncp"]) == tuple(bs.ncp[b]) and tuple(d["degree"]) == tuple(bs.degree[b])
        assert tuple(d["nsamp"]) == (16, 16, 16) and d["slot"] == i
        C, p = bs.ncp[b, 0], bs.degree[b, 0]
        for a in range(3):
            want = bs.knots[bs.knot_off[b, a]: bs.knot_off[b, a] + C + p + 1]
            assert np.array_equal(knots[d["knot_off"][a]: d["knot_off"][a] + C + p + 1], want)
        assert np.array_equal(cps[d["cp_off"]: d["cp_off"] + C ** 3], bs.cps[bs.cp_off[b]: bs.cp_off[b] + C ** 3])
    assert batch.bounds.max_ncp == bs.ncp[ids].max() and batch.bounds.max_nsamp == 16
    with pytest.raises(mfa.MfaError):
        cache.upload([1], 16, batch)  # not cached
    cache.close()


@pytest.mark.parametrize("apron", [True, False])
def test_out_of_core_frames_equal_in_core_frames(mfa, ctx, tmp_path, apron):
    """128^3 flame, 512 bricks of 16^3 (C in {4, 6, 8, 12}); 6 orbit frames through a 200-model cache with
    prefetching of the extrapolated next view (slots in the apron or the row layout), against decode + ray
    cast of the resident models in the row layout."""
    from paper_2409_00184_b300.outofcore import OutOfCoreRenderer, extrapolate_view
    N, n, p = 128, 16, 2
    bs, B = flame_blockset(N, n, (4, 6, 8, 12), (50, 75, 90), p, synth.BASE_SEED + 3, "cpu")
    path = tmp_path / "flame.mfa"
    mfa.store_write(path, bs)
    tf = torch.from_numpy(synth.transfer_function(synth.BASE_SEED + 3)).cuda()
    fov = synth.fov_for_visible(110, B)
    views = [synth.orbit_view(f, fov_y_deg=fov, width=48, height=40) for f in range(6)]
    vis = [synth.visible_bricks(v, B) for v in views]
    assert max(len(v) for v in vis) <= 200
    ooc = OutOfCoreRenderer(ctx, path, 200, (B, B, B), n, tf, 48, 40, apron=apron)
    blk = mfa.DeviceBlocks(bs)
    cache = torch.empty(200 * n ** 3 * 4, device="cuda")
    table = torch.full((B, B, B), -1, dtype=torch.int32, device="cuda")
    ref = torch.zeros(40, 48, 4, device="cuda")
    stats = []
    for f, v in enumerate(views):
        pred = None
        if f >= 1:
            pred = synth.visible_bricks(extrapolate_view(views[f - 1], v), B)
        stats.append(ooc.frame(vis[f], v, predicted=pred))
        got = ooc.image.clone()
        lst = torch.from_numpy(vis[f]).cuda()
        mfa.decode_blocks(ctx, blk, cache, n ** 3, len(vis[f]), list_=lst, flags=mfa.DECODE_LIST_SLOTS)
        tab = np.full(B ** 3, -1, np.int32)
        tab[vis[f]] = np.arange(len(vis[f]), dtype=np.int32)
        table.copy_(torch.from_numpy(tab.reshape(B, B, B)))
        mfa.raycast(ctx, cache, n ** 3, len(vis[f]), table, n, v, tf, ref)
        assert ctx.device_status() == 0
        assert torch.equal(got, ref), f
    ooc.close()
    assert stats[0]["misses"] == len(vis[0]) and stats[0]["hits"] == 0
    assert all(s["hits"] > 0 for s in stats[1:])
    assert sum(s["prefetched"] for s in stats) > 0
