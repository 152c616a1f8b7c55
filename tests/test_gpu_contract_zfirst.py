"""The z-first contraction kernel (the least-squares fit without its RMSE pass, and the adjoint, for blocks
of at most 32 samples and 16 control points per axis) against the FP64 oracle. Batches mix 32x32-plane
blocks (loaded by TMA) with blocks whose x-rows or y-columns are shorter (copied into shared memory),
several classes and degrees in one launch, more blocks than CTAs (the slab ring runs from block to block
and set-ups are reused or rebuilt), and blocks that fail their device-side checks."""

import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj
from oracle import encode

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


def _batch(B, seed, shapes):
    """B blocks cycling through `shapes` = [(C, p, (nx, ny, nz)), ...]; random sample grids in [-1, 1]."""
    ncp, deg, ns = [], [], []
    for b in range(B):
        C, p, n = shapes[b % len(shapes)]
        ncp.append((C,) * 3), deg.append((p,) * 3), ns.append(n)
    bs = synth.make_block_set(ncp, deg, ns, [np.zeros((C[2], C[1], C[0])) for C in ncp])
    g = synth.rng(seed)
    stride = int(np.max(np.prod(bs.nsamp.astype(np.int64), axis=1)))
    stride = (stride + 31) // 32 * 32  # slots hold whole rows of 32: the TMA path
    grids = np.zeros((B, stride), np.float32)
    for b in range(B):
        nx, ny, nz = bs.nsamp[b]
        grids[b, : nx * ny * nz] = g.uniform(-1, 1, nx * ny * nz)
    return bs, grids, stride


def _grid(grids, bs, b):
    nx, ny, nz = bs.nsamp[b]
    return grids[bs.slot[b], : nx * ny * nz].reshape(nz, ny, nx).astype(np.float64)


def _cps(out, bs, b):
    Cx, Cy, Cz = bs.ncp[b]
    return out[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)


SHAPES = [(8, 2, (32, 32, 32)), (12, 2, (32, 32, 32)), (12, 3, (32, 32, 32)), (16, 2, (32, 32, 32)),
          (4, 1, (32, 32, 32)), (6, 2, (32, 24, 32)), (8, 3, (16, 32, 20)), (5, 2, (13, 8, 32))]


@pytest.mark.parametrize("B", [len(SHAPES), 300])
def test_zfirst_adjoint_matches_oracle(mfa, ctx, B):
    bs, R, stride = _batch(B, 700 + B, SHAPES)
    blk = mfa.DeviceBlocks(bs)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, B, grad)
    assert ctx.device_status() == 0
    G = grad.cpu().numpy()
    assert np.isfinite(G).all()
    check = range(B) if B <= 16 else sorted(set(synth.rng(3).choice(B, 14, replace=False).tolist()) | {0, B - 1})
    for b in check:
        want = oadj.adjoint_block(_grid(R, bs, b), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        assert np.abs(_cps(G, bs, b) - want).max() <= 1e-5 * np.abs(want).max(), b


@pytest.mark.parametrize("B", [len(SHAPES), 300])
def test_zfirst_fit_matches_oracle(mfa, ctx, B):
    bs, D, stride = _batch(B, 710 + B, SHAPES)
    blk = mfa.DeviceBlocks(bs)
    plan = mfa.EncodePlan(ctx, blk)
    out = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.encode_blocks(ctx, plan, torch.from_numpy(D.ravel()).cuda(), stride, B, out)  # no RMSE: z-first kernel
    assert ctx.device_status() == 0
    P = out.cpu().numpy()
    assert np.isfinite(P).all()
    check = range(B) if B <= 16 else sorted(set(synth.rng(4).choice(B, 14, replace=False).tolist()) | {0, B - 1})
    for b in check:
        want = encode.fit_separable(_grid(D, bs, b), bs.block_knots(b), bs.degree[b])
        assert np.abs(_cps(P, bs, b) - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), b


def test_zfirst_fit_equals_the_fit_with_rmse(mfa, ctx):
    """The fit with its RMSE pass runs on the slab kernel (x first), this one z first: both are within the
    oracle tolerance of the same least-squares control points, so they agree to that tolerance."""
    bs, D, stride = _batch(40, 720, SHAPES)
    blk = mfa.DeviceBlocks(bs)
    plan = mfa.EncodePlan(ctx, blk)
    d = torch.from_numpy(D.ravel()).cuda()
    a = torch.empty(blk.cps_len, device="cuda")
    b = torch.empty(blk.cps_len, device="cuda")
    rm = torch.empty(40, dtype=torch.float64, device="cuda")
    mfa.encode_blocks(ctx, plan, d, stride, 40, a)
    mfa.encode_blocks(ctx, plan, d, stride, 40, b, rm)
    assert ctx.device_status() == 0
    scale = max(1.0, float(b.abs().max()))
    assert float((a - b).abs().max()) <= 1e-5 * scale


def test_zfirst_skips_blocks_that_fail_their_checks(mfa, ctx):
    """300 blocks on at most 148 CTAs: blocks 150 and 151 sit between blocks 2 / 298 and 3 / 299 in their
    CTAs' streams (block b goes to CTA b mod grid), so a skipped block must leave the ring and the set-up
    buffers consistent for the blocks after it."""
    B = 300
    bs, R, stride = _batch(B, 730, SHAPES[:4])
    # block 150 (TMA-fed): decreasing knots on x; block 151: slot out of range
    kn = np.array(bs.block_knots(150)[0][::-1], dtype=np.float32)
    bs.knot_off[150, 0] = len(bs.knots)
    bs.knots = np.concatenate([bs.knots, kn])
    bs.slot[151] = 999
    blk = mfa.DeviceBlocks(bs)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, B, grad)
    st = ctx.device_status()
    assert st & mfa.DEV_BAD_KNOTS and st & mfa.DEV_BAD_RANGE
    G = grad.cpu().numpy()
    assert np.isnan(_cps(G, bs, 150)).all() and np.isnan(_cps(G, bs, 151)).all()
    for b in (0, 2, 3, 149, 152, 298, 299):
        want = oadj.adjoint_block(_grid(R, bs, b), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        assert np.abs(_cps(G, bs, b) - want).max() <= 1e-5 * np.abs(want).max(), b
    assert ctx.device_status() == 0


def test_zfirst_adjoint_at_the_step_size_sampled():
    """The adjoint as the 512^3 step launches it: 4096 blocks of 32^3, C = 12, degree 2, on the z-first kernel
    (one CTA per SM, about 28 blocks each, so the set-up buffers rotate many times), over the step's own
    synthetic field as the residual; 18 sampled blocks (the first and last among them) against the FP64
    oracle's adjoint."""
    from paper_2409_00184_b300 import mfa
    torch.cuda.set_device(0)
    ctx = mfa.Context(0)
    N, n, C, p = 512, 32, 12, 2
    field = synth.gm_noise_field(N, synth.BASE_SEED + 2, device="cuda")
    R = synth.blocks_from_field(field, n).contiguous().view(-1)
    del field
    B = (N // n) ** 3
    bs = synth.make_block_set([(C,) * 3] * B, [(p,) * 3] * B, [(n,) * 3] * B, [np.zeros((C, C, C))] * B)
    blk = mfa.DeviceBlocks(bs)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, R, n ** 3, B, grad)
    assert ctx.device_status() == 0
    G = grad.view(B, C ** 3)
    assert bool(torch.isfinite(G).all())
    pick = sorted(set(synth.rng(5).choice(B, 16, replace=False).tolist()) | {0, B - 1})
    Rv = R.view(B, n, n, n)
    for b in pick:
        want = oadj.adjoint_block(Rv[b].double().cpu().numpy(), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        got = G[b].double().cpu().numpy().reshape(C, C, C)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), b
    ctx.close()
