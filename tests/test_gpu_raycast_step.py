"""The ray cast of the benchmarked step against the oracle's Algorithm 4 on sampled pixels.

512^3 Gaussian-mixture + noise field, 4096 bricks of 32^3 (degree 2, 12^3 control points), decoded into
the apron layout, apron planes filled, and ray-cast at 1024^2 with early termination (O_max = 0.99) by
the persistent queue kernel: the launch sequence and sizes of the step. The control points are the
oracle's least-squares fit of the field's blocks, so that the decode and the ray cast are compared on the
same models; the oracle marches 2000 seeded rays over nodes it decodes on demand.
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import node_groups, oracle_fit_all
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


def _compare(got, want):
    d = np.abs(got - want).max(axis=-1)
    return d, float(d.max()), float((d <= 1e-4).mean())


def test_step_raycast_full_size_sampled_pixels(mfa, ctx):
    N, n, C, p, img = 512, 32, 12, 2, 1024
    seed = synth.BASE_SEED + 2
    field = synth.gm_noise_field(N, seed, device="cuda")
    Dd = synth.blocks_from_field(field, n).contiguous()
    del field
    B = Dd.shape[0]
    P = oracle_fit_all(Dd.cpu().numpy(), C, p)
    bs = synth.make_block_set([(C,) * 3] * B, [(p,) * 3] * B, [(n,) * 3] * B, list(P))
    blk = mfa.DeviceBlocks(bs)
    S = mfa.apron_voxels(n)
    cache = torch.empty(B * S * 4, device="cuda")
    R = torch.empty(B * n ** 3, device="cuda")
    rm = torch.empty(B, dtype=torch.float64, device="cuda")
    nb = N // n
    table = torch.arange(B, dtype=torch.int32, device="cuda").view(nb, nb, nb)
    tf = synth.transfer_function(seed)
    view = synth.default_view(img, img)
    image = torch.full((img, img, 4), float("nan"), device="cuda")
    mfa.decode_compare_blocks(ctx, blk, cache, S, B, Dd.view(-1), n ** 3, residual=R, rmse=rm, flags=mfa.DECODE_APRON)
    mfa.fill_aprons(ctx, cache, S, B, table, n)
    mfa.raycast(ctx, cache, S, B, table, n, view, torch.from_numpy(tf).cuda(), image, apron=True)
    assert ctx.device_status() == 0
    got = image.view(-1, 4).cpu().numpy()
    assert not np.isnan(got).any()
    del cache, R
    pix = synth.rng(71).choice(img * img, 2000, replace=False)
    voxels = ocast.decoded_nodes(node_groups(bs), B)
    want = ocast.raycast(voxels, table.cpu().numpy(), n, view, tf, pixels=pix)
    d, dmax, within = _compare(got[pix], want)
    print(f"step ray cast, 2000 pixels: max {dmax:.2e}, within 1e-4: {within:.4f}, "
          f"opaque: {(want[:, 3] > 0.99).mean():.3f}, lit: {(want[:, 3] > 0).mean():.3f}")
    assert (want[:, 3] > 0).mean() > 0.3  # the sample sees the volume
    assert dmax <= 1e-2 and within >= 0.999
