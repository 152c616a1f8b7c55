"""Levels of detail and cross-level adaptive encoding (Sec. 4.2.3, Algorithm 1) on the GPU against the FP64
oracle: the LOD partition bit for bit, and the per-level search sets, simple/complex decisions, NCP* and
RMSE of the final per-block encode."""

import numpy as np
import pytest
import torch

import synth
from oracle import encode as oenc

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


@pytest.mark.parametrize("stride", [1, 2, 4])
def test_lod_gather_matches_oracle(mfa, ctx, stride):
    g = synth.rng(900 + stride)
    F = g.uniform(-1, 1, (48, 32, 64)).astype(np.float32)  # (Nz, Ny, Nx), anisotropic
    n = 4
    want, B = oenc.lod_blocks(F, n, stride)
    got = mfa.lod_gather(ctx, torch.from_numpy(F).cuda(), n, stride).cpu().numpy()
    assert got.shape == (B[0] * B[1] * B[2], n ** 3)
    assert np.array_equal(got, want.reshape(len(want), -1))
    ids = torch.as_tensor(g.permutation(len(want))[:7].astype(np.int32)).cuda()
    sub = mfa.lod_gather(ctx, torch.from_numpy(F).cuda(), n, stride, ids=ids).cpu().numpy()
    assert np.array_equal(sub, want.reshape(len(want), -1)[ids.cpu().numpy()])
    assert ctx.device_status() == 0


def test_lod_gather_checks(mfa, ctx):
    F = torch.zeros(16, 16, 16, device="cuda")
    with pytest.raises(mfa.MfaError):
        mfa.lod_gather(ctx, F, 3, 2)  # 16 is not a multiple of 6
    bad = torch.tensor([0, 9], dtype=torch.int32, device="cuda")  # the level has 8 blocks
    out = torch.full((2, 64), 7.0, device="cuda")
    mfa.lod_gather(ctx, F, 4, 2, ids=bad, out=out)
    assert ctx.device_status() == mfa.DEV_BAD_LIST
    assert (out[1] == 7.0).all() and (out[0] == 0.0).all()


def test_cross_level_encode_matches_oracle():
    """64^3 flame stand-in, micro-blocks of 8^3, degree 2, 3 levels (2^3, 4^3, 8^3 blocks), RMSE bound 1.5e-2
    (every candidate RMSE of the oracle is at least 1.6e-4 away from it, so every decision is unique)."""
    from paper_2409_00184_b300 import adaptive, mfa
    ctx = mfa.Context(0)
    n, p, bound, levels = 8, 2, 1.5e-2, 3
    field = synth.flame_field(64, synth.BASE_SEED + 16, device="cuda")
    F = field.double().cpu().numpy()
    want = oenc.cross_level_select(F, n, p, bound, levels)
    got = adaptive.cross_level_encode(ctx, field, n, p, bound, levels)
    assert ctx.device_status() == 0
    assert [r["level"] for r in got] == [r["level"] for r in want]
    for gr, wr in zip(got, want):
        assert np.array_equal(gr["searched"], wr["searched"]), gr["level"]
        assert np.array_equal(gr["complex"], wr["complex"]), gr["level"]
        assert np.array_equal(gr["ncp"], wr["ncp"]), gr["level"]
        # the final encode with the chosen per-block NCP: RMSE against the oracle's fit of the same block
        blocks, _ = oenc.lod_blocks(F, n, gr["stride"])
        rm = gr["rmse"].cpu().numpy()
        for b in synth.rng(17).choice(len(blocks), min(12, len(blocks)), replace=False):
            C = int(gr["ncp"][b])
            t = np.float32(synth.clamped_uniform_knots(C, p)).astype(np.float64)
            P = oenc.fit_separable(blocks[b], (t, t, t), (p, p, p))
            assert abs(rm[b] - oenc.rmse(P, blocks[b], (t, t, t), (p, p, p))) <= 1e-5 * (F.max() - F.min())
    searched = sum(int(r["searched"].sum()) for r in got)
    assert 0 < searched < sum(len(r["ncp"]) for r in got)  # the cross-level rule skipped some blocks
    assert any((r["searched"] & ~r["complex"]).any() for r in got)
    ctx.close()
