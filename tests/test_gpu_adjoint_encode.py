"""GPU adjoint (mfa_adjoint_blocks) and least-squares encode (mfa_encode_blocks) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted
from oracle import adjoint as oadj
from oracle import decode, encode

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


def _grids(bs, seed):
    g = synth.rng(seed)
    stride = int(np.max(np.prod(bs.nsamp.astype(np.int64), axis=1)))
    grids = np.zeros((len(bs), stride), np.float32)
    for b in range(len(bs)):
        nx, ny, nz = bs.nsamp[b]
        grids[bs.slot[b], : nx * ny * nz] = g.uniform(-1, 1, nx * ny * nz)
    return grids, stride


def _block_grid(grids, bs, b):
    nx, ny, nz = bs.nsamp[b]
    return grids[bs.slot[b], : nx * ny * nz].reshape(nz, ny, nx).astype(np.float64)


@pytest.mark.parametrize("seed", [301, 302])
def test_adjoint_matches_oracle(mfa, ctx, seed):
    bs = synth.random_block_set(16, seed, nsamp_choices=(5, 13, 32, 64), ncp_choices=(4, 6, 8, 12, 20),
                                nonuniform=seed % 2 == 0)
    blk = mfa.DeviceBlocks(bs)
    R, stride = _grids(bs, seed)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, len(bs), grad)
    assert ctx.device_status() == 0
    G = grad.cpu().numpy()
    for b in range(len(bs)):
        want = oadj.adjoint_block(_block_grid(R, bs, b), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), b


def test_fused_residual_gradient(mfa, ctx):
    bs = synth.random_block_set(12, 303, nsamp_choices=(8, 13, 32), ncp_choices=(4, 6, 8))
    blk = mfa.DeviceBlocks(bs)
    D, stride = _grids(bs, 303)
    grad = torch.zeros(blk.cps_len, device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(D.ravel()).cuda(), stride, len(bs), grad, cps=blk.cps)
    assert ctx.device_status() == 0
    G = grad.cpu().numpy()
    for b in range(len(bs)):
        knots, deg, nsamp = bs.block_knots(b), bs.degree[b], bs.nsamp[b]
        r = decode.decode_block(bs.block_cps(b), knots, deg, nsamp)[..., 0] - _block_grid(D, bs, b)
        want = oadj.adjoint_block(r, knots, deg, bs.ncp[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), b


def _encode(mfa, ctx, bs, D, stride):
    blk = mfa.DeviceBlocks(bs)
    plan = mfa.EncodePlan(ctx, blk)
    out = torch.full((blk.cps_len,), float("nan"), device="cuda")
    rmse = torch.full((len(bs),), float("nan"), dtype=torch.float64, device="cuda")
    mfa.encode_blocks(ctx, plan, torch.from_numpy(np.ascontiguousarray(D).ravel()).cuda(), stride, len(bs), out, rmse)
    assert ctx.device_status() == 0
    plan.close()
    return out.cpu().numpy(), rmse.cpu().numpy()


@pytest.mark.parametrize("seed,nonuniform", [(311, False), (312, True)])
def test_encode_matches_oracle_least_squares(mfa, ctx, seed, nonuniform):
    # non-uniform knots keep every span at least one sample spacing wide (a well-posed fit)
    bs = synth.random_block_set(16, seed, nsamp_choices=(13, 32, 64), ncp_choices=(3, 4, 6, 8, 12) if nonuniform
                                else (3, 4, 6, 8, 12, 16, 24), nonuniform=nonuniform, min_gap=0.085)
    D, stride = _grids(bs, seed)
    P, rm = _encode(mfa, ctx, bs, D, stride)
    for b in range(len(bs)):
        Db = _block_grid(D, bs, b)
        want = encode.fit_separable(Db, bs.block_knots(b), bs.degree[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = P[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), b
        want_rmse = encode.rmse(want, Db, bs.block_knots(b), bs.degree[b])
        assert abs(rm[b] - want_rmse) <= 1e-5 * (Db.max() - Db.min()), (b, rm[b], want_rmse)


def test_encode_gm_128cubed_c12_degree2(mfa, ctx):
    bs, blocks = gm_blocks_fitted(128, 32, 12, 2, synth.BASE_SEED + 2)
    D = blocks.reshape(len(bs), -1)
    P, rm = _encode(mfa, ctx, bs, D, 32 ** 3)
    want = bs.cps.astype(np.float64)  # the oracle's least-squares control points
    rng_p = want.max() - want.min()
    assert np.abs(P - want).max() <= 1e-5 * rng_p
    assert np.all(rm > 0) and np.all(rm < 0.05)


def test_encode_plan_rejects_bad_batches(mfa, ctx):
    bs = synth.random_block_set(2, 313, ncp_choices=(12,), nsamp_choices=(8,), degree_choices=(2,))
    bs.ncp[:] = 12  # C > n: not a least-squares problem with a unique solution
    blk = mfa.DeviceBlocks(bs)
    with pytest.raises(mfa.MfaError) as e:
        mfa.EncodePlan(ctx, blk)
    assert e.value.code == mfa.ERR_INVALID_ARG


@pytest.mark.parametrize("flags_name", ["", "VALUE_ONLY"])
def test_decode_compare_fuses_residual_and_rmse(mfa, ctx, flags_name):
    """mfa_decode_compare_blocks: the cache equals mfa_decode_blocks', the residual equals decode(P) - D, and
    the RMSE equals both the fit's RMSE (same fitted P) and the oracle's, on fitted Gaussian-mixture blocks
    and on a ragged random batch through a device-counted list with list slots."""
    flags = getattr(mfa, "DECODE_" + flags_name) if flags_name else 0
    width = 1 if flags_name else 4
    # fitted blocks: the fit's RMSE is the reference
    bs, blocks = gm_blocks_fitted(64, 16, 8, 2, synth.BASE_SEED + 20)
    blk = mfa.DeviceBlocks(bs)
    nb, vox = len(bs), 16 ** 3
    D = torch.from_numpy(blocks.reshape(-1)).cuda()
    plan = mfa.EncodePlan(ctx, blk)
    fit_rmse = torch.empty(nb, dtype=torch.float64, device="cuda")
    mfa.encode_blocks(ctx, plan, D, vox, nb, blk.cps, fit_rmse)
    plan.close()
    cache_a = torch.zeros(nb * vox * width, device="cuda")
    cache_b = torch.zeros(nb * vox * width, device="cuda")
    res = torch.full((nb * vox,), float("nan"), device="cuda")
    rm = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
    mfa.decode_blocks(ctx, blk, cache_a, vox, nb, flags=flags)
    mfa.decode_compare_blocks(ctx, blk, cache_b, vox, nb, D, vox, residual=res, rmse=rm, flags=flags)
    assert ctx.device_status() == 0
    assert torch.equal(cache_a, cache_b)
    f = cache_b.view(nb, vox, width)[:, :, 0]
    assert torch.equal(res.view(nb, vox), f - D.view(nb, vox))
    drange = float(blocks.max() - blocks.min())
    assert float((rm - fit_rmse).abs().max()) <= 1e-6 * drange
    for b in range(0, nb, 9):
        P = bs.block_cps(b)
        want = encode.rmse(P, blocks[b].astype(np.float64), bs.block_knots(b), tuple(bs.degree[b]))
        assert abs(float(rm[b]) - want) <= 1e-5 * drange
    # ragged batch, list with a device count and list slots
    rb = synth.random_block_set(14, 321, nsamp_choices=(5, 13, 32), ncp_choices=(4, 6))
    rblk = mfa.DeviceBlocks(rb)
    Dr, stride = _grids(rb, 321)
    lst = torch.tensor([3, 11, 0, 7, 5], dtype=torch.int32, device="cuda")
    cnt = torch.tensor([4], dtype=torch.int32, device="cuda")
    Dl = torch.from_numpy(np.ascontiguousarray(Dr[rb.slot[lst.cpu().numpy()]]).ravel()).cuda()  # slot m: item m
    cache = torch.zeros(5 * stride * width, device="cuda")
    rml = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    mfa.decode_compare_blocks(ctx, rblk, cache, stride, 5, Dl, stride, rmse=rml, flags=flags | mfa.DECODE_LIST_SLOTS,
                              list_=lst, count=cnt)
    assert ctx.device_status() == 0
    got = rml.cpu().numpy()
    for m, b in enumerate(lst.cpu().numpy()[:4]):
        nx, ny, nz = rb.nsamp[b]
        g = Dl[m * stride: m * stride + nx * ny * nz].double().cpu().numpy().reshape(nz, ny, nx)
        want = encode.rmse(rb.block_cps(b), g, rb.block_knots(b), tuple(rb.degree[b]))
        assert abs(got[m] - want) <= 1e-5 * max(1.0, float(np.abs(g).max())), (m, b)
    assert got[4] == 0.0  # beyond the device count: zeroed, not decoded


def test_repeated_interior_knots_adjoint_and_fit(mfa, ctx):
    """Knot vectors with repeated interior knots (multiplicity up to p, so spans skip empty intervals and a
    band can move by several control points between samples): the adjoint and the least-squares fit (with its
    RMSE pass, and without it on the z-first kernel where the shapes allow) against the FP64 oracle."""
    from gpu_util import repeated_knot_set
    bs = repeated_knot_set(10, 341, nsamp_choices=(13, 32))
    blk = mfa.DeviceBlocks(bs)
    R, stride = _grids(bs, 342)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, len(bs), grad)
    assert ctx.device_status() == 0
    G = grad.cpu().numpy()
    for b in range(len(bs)):
        want = oadj.adjoint_block(_block_grid(R, bs, b), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), b
    # the fit, on 32 samples per axis (every span of these knots holds samples: a well-posed fit)
    fb = repeated_knot_set(8, 343, nsamp_choices=(32,))
    D, stride = _grids(fb, 344)
    P, rm = _encode(mfa, ctx, fb, D, stride)
    fblk = mfa.DeviceBlocks(fb)
    plan = mfa.EncodePlan(ctx, fblk)
    Pz = torch.full((fblk.cps_len,), float("nan"), device="cuda")
    mfa.encode_blocks(ctx, plan, torch.from_numpy(np.ascontiguousarray(D).ravel()).cuda(), stride, len(fb), Pz)
    assert ctx.device_status() == 0
    plan.close()
    Pz = Pz.cpu().numpy()
    for b in range(len(fb)):
        Db = _block_grid(D, fb, b)
        want = encode.fit_separable(Db, fb.block_knots(b), fb.degree[b])
        Cx, Cy, Cz = fb.ncp[b]
        for got in (P, Pz):
            g = got[fb.cp_off[b]: fb.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
            assert np.abs(g - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), b
        want_rmse = encode.rmse(want, Db, fb.block_knots(b), fb.degree[b])
        assert abs(rm[b] - want_rmse) <= 1e-5 * (Db.max() - Db.min()), (b, rm[b], want_rmse)


def test_smallest_blocks_decode_adjoint_fit(mfa, ctx):
    """The smallest blocks the library takes: 2 or 3 samples per axis with C = p + 1 <= n control points
    (degree 1 or 2, a single Bezier span). The FP32 decode, the adjoint and the least-squares fit (with
    C = n the fit interpolates the samples) against the FP64 oracle."""
    specs = [((2, 2, 2), (1, 1, 1), (2, 2, 2)), ((3, 3, 3), (2, 2, 2), (3, 3, 3)), ((2, 3, 2), (1, 2, 1), (3, 3, 2)),
             ((2, 2, 3), (1, 1, 2), (2, 3, 3))]
    g = synth.rng(361)
    ncp, deg, ns, cps = [], [], [], []
    for C, p, n in specs * 2:
        ncp.append(C), deg.append(p), ns.append(n)
        cps.append(g.uniform(-1, 1, (C[2], C[1], C[0])))
    bs = synth.make_block_set(ncp, deg, ns, cps)
    blk = mfa.DeviceBlocks(bs)
    V = blk.slot_voxels
    cache = torch.full((len(bs) * V * 4,), float("nan"), device="cuda")
    mfa.decode_blocks(ctx, blk, cache, V, len(bs))
    R, stride = _grids(bs, 362)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, len(bs), grad)
    assert ctx.device_status() == 0
    c = cache.view(len(bs), V, 4).cpu().numpy()
    G = grad.cpu().numpy()
    for b in range(len(bs)):
        nx, ny, nz = bs.nsamp[b]
        Cx, Cy, Cz = bs.ncp[b]
        want = decode.decode_block(bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b])
        got = c[bs.slot[b], : nx * ny * nz].reshape(nz, ny, nx, 4)
        assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), b
        gw = oadj.adjoint_block(_block_grid(R, bs, b), bs.block_knots(b), bs.degree[b], bs.ncp[b])
        gg = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(gg - gw).max() <= 1e-5 * max(1e-30, np.abs(gw).max()), b
    D, stride = _grids(bs, 363)
    P, rm = _encode(mfa, ctx, bs, D, stride)
    for b in range(len(bs)):
        Db = _block_grid(D, bs, b)
        want = encode.fit_separable(Db, bs.block_knots(b), bs.degree[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = P[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), b
        assert abs(rm[b] - encode.rmse(want, Db, bs.block_knots(b), bs.degree[b])) <= 1e-5 * (Db.max() - Db.min())
