"""Tensor-core (tcgen05) fit and adjoint in split-BF16 and BF16 against the FP64 oracle.

mfa_adjoint_blocks and mfa_encode_blocks_ex with MFA_PREC_SPLIT_BF16 / MFA_PREC_BF16: 32 samples and at most
16 control points per axis. Tolerances (relative to the largest |output| for the adjoint, to the range of
the control points for the fit): split-BF16 1e-4, BF16 1e-2 (adjoint) and 5e-2 (fit). Also: gradient descent with the split-BF16
gradient reaches 1e-4 of the FP64 least-squares solve (256^3 field, 512 blocks, C in {8, 12, 16}).
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import gm_blocks_fitted
from oracle import adjoint as oadj
from oracle import encode as oenc

pytestmark = pytest.mark.gpu

TOL = {"split": 1e-4, "bf16": 1e-2}
# Plain BF16 fit: the pseudo-inverses are dense with mixed signs, so each of the three stages rounds its
# operands to 2^-9 relative and the next stages amplify that by the pseudo-inverse's row 1-norm (about 2.2 at
# C = 12): 3 * 2^-9 * 2.2^2 ~ 3e-2 of the control points' range.
TOL_FIT = {"split": 1e-4, "bf16": 5e-2}


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
    return {"split": mfa.PREC_SPLIT_BF16, "bf16": mfa.PREC_BF16}[name]


def _grids(bs, seed, stride):
    g = synth.rng(seed)
    grids = np.zeros((len(bs), stride), np.float32)
    for b in range(len(bs)):
        grids[bs.slot[b], : 32 ** 3] = g.uniform(-1, 1, 32 ** 3)
    return grids


@pytest.mark.parametrize("name", ["split", "bf16"])
@pytest.mark.parametrize("nonuniform", [False, True])
def test_tc_adjoint_matches_oracle(mfa, ctx, name, nonuniform):
    bs = synth.random_block_set(40, 701 + nonuniform, nsamp_choices=(32,), ncp_choices=(2, 3, 4, 7, 12, 16),
                                degree_choices=(1, 2, 3), nonuniform=nonuniform, min_gap=0.05)
    blk = mfa.DeviceBlocks(bs)
    stride = 32 ** 3 + 64  # slots further apart than one grid
    R = _grids(bs, 702, stride)
    grad = torch.full((blk.cps_len,), float("nan"), device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), stride, len(bs), grad, precision=_prec(mfa, name))
    assert ctx.device_status() == 0
    G = grad.cpu().numpy()
    worst = 0.0
    for b in range(len(bs)):
        Rb = R[bs.slot[b], : 32 ** 3].reshape(32, 32, 32).astype(np.float64)
        want = oadj.adjoint_block(Rb, bs.block_knots(b), bs.degree[b], bs.ncp[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    print(f"{name} adjoint, nonuniform={nonuniform}: {worst:.2e}")
    assert worst <= TOL[name]


@pytest.mark.parametrize("name", ["split", "bf16"])
def test_tc_fit_matches_oracle(mfa, ctx, name):
    """Gaussian-mixture blocks (128^3 field, 64 blocks of 32^3) at C = 12 and degree 2, and a mixed batch of
    C in {4, 8, 16} with degrees 1..3, against the oracle's separable least squares."""
    for bs, D in (gm_blocks_fitted(128, 32, 12, 2, synth.BASE_SEED + 30),
                  _mixed_fit_batch()):
        D = np.asarray(D, np.float32).reshape(len(bs), -1)
        blk = mfa.DeviceBlocks(bs)
        plan = mfa.EncodePlan(ctx, blk)
        out = torch.full((blk.cps_len,), float("nan"), device="cuda")
        mfa.encode_blocks(ctx, plan, torch.from_numpy(D.ravel()).cuda(), 32 ** 3, len(bs), out,
                          precision=_prec(mfa, name))
        assert ctx.device_status() == 0
        plan.close()
        P = out.cpu().numpy()
        worst = 0.0
        for b in range(len(bs)):
            want = oenc.fit_separable(D[bs.slot[b]].reshape(32, 32, 32).astype(np.float64), bs.block_knots(b),
                                      bs.degree[b])
            Cx, Cy, Cz = bs.ncp[b]
            got = P[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
            worst = max(worst, np.abs(got - want).max() / max(1e-12, want.max() - want.min()))
        print(f"{name} fit ({len(bs)} blocks): {worst:.2e}")
        assert worst <= TOL_FIT[name]


def _mixed_fit_batch():
    bs = synth.random_block_set(24, 711, nsamp_choices=(32,), ncp_choices=(4, 8, 16), degree_choices=(1, 2, 3))
    D = synth.rng(712).uniform(-1, 1, (len(bs), 32 ** 3)).astype(np.float32)
    return bs, D


def test_tc_paths_refuse_what_they_do_not_cover(mfa, ctx):
    bs = synth.random_block_set(4, 721, nsamp_choices=(32,), ncp_choices=(20,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    R = torch.zeros(len(bs) * 32 ** 3, device="cuda")
    G = torch.zeros(blk.cps_len, device="cuda")
    with pytest.raises(mfa.MfaError) as e:  # C = 20 > 16
        mfa.adjoint_blocks(ctx, blk, R, 32 ** 3, len(bs), G, precision=mfa.PREC_SPLIT_BF16)
    assert e.value.code == mfa.ERR_UNSUPPORTED
    bs2 = synth.random_block_set(4, 722, nsamp_choices=(32,), ncp_choices=(8,), degree_choices=(2,))
    blk2 = mfa.DeviceBlocks(bs2)
    G2 = torch.zeros(blk2.cps_len, device="cuda")
    with pytest.raises(mfa.MfaError) as e:  # the fused gradient stays FP32
        mfa.adjoint_blocks(ctx, blk2, R, 32 ** 3, len(bs2), G2, cps=blk2.cps, precision=mfa.PREC_SPLIT_BF16)
    assert e.value.code == mfa.ERR_UNSUPPORTED
    plan = mfa.EncodePlan(ctx, blk2)
    rm = torch.zeros(len(bs2), dtype=torch.float64, device="cuda")
    with pytest.raises(mfa.MfaError) as e:  # the RMSE pass stays FP32
        mfa.encode_blocks(ctx, plan, R, 32 ** 3, len(bs2), G2, rm, precision=mfa.PREC_SPLIT_BF16)
    assert e.value.code == mfa.ERR_UNSUPPORTED
    with pytest.raises(mfa.MfaError) as e:
        mfa.adjoint_blocks(ctx, blk2, R, 32 ** 3, len(bs2), G2, precision=mfa.PREC_FP16)
    assert e.value.code == mfa.ERR_UNSUPPORTED
    plan.close()
    assert ctx.device_status() == 0
    # no blocks: the call returns before any check of the (absent) arrays and launches nothing
    import ctypes
    n0 = ctx.launch_count()
    for prec in (mfa.PREC_SPLIT_BF16, mfa.PREC_BF16):
        rc = mfa.lib.mfa_adjoint_blocks(ctx.handle, None, 0, None, 0, None, 32 ** 3, 0, None, None, 0,
                                        ctypes.byref(blk2.bounds), prec,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == mfa.OK
    assert ctx.launch_count() == n0


def test_tc_adjoint_skips_a_block_of_another_shape(mfa, ctx):
    """A block with 16 samples on one axis in a batch bounded by 32 sets MFA_DEV_BAD_DESC and is skipped; the
    others are exact."""
    bs = synth.random_block_set(6, 731, nsamp_choices=(32,), ncp_choices=(6, 8), degree_choices=(2,))
    bs.nsamp[3, 1] = 16
    blk = mfa.DeviceBlocks(bs)
    R = _grids(bs, 732, 32 ** 3)
    grad = torch.full((blk.cps_len,), -7.0, device="cuda")
    mfa.adjoint_blocks(ctx, blk, torch.from_numpy(R.ravel()).cuda(), 32 ** 3, len(bs), grad,
                       precision=mfa.PREC_SPLIT_BF16)
    assert ctx.device_status() == mfa.DEV_BAD_DESC
    G = grad.cpu().numpy()
    for b in range(len(bs)):
        Cx, Cy, Cz = bs.ncp[b]
        got = G[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz]
        if b == 3:
            assert np.all(got == -7.0)
            continue
        Rb = R[bs.slot[b]].reshape(32, 32, 32).astype(np.float64)
        want = oadj.adjoint_block(Rb, bs.block_knots(b), bs.degree[b], bs.ncp[b]).ravel()
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()


def test_gradient_descent_split_bf16_256cubed_512_blocks(mfa, ctx):
    """Split-BF16 gradient descent on the 256^3 field, 512 blocks of 32^3, C in {8, 12, 16} by gradient-energy
    terciles; Nesterov descent with the split-BF16 tensor-core adjoint until max|P - P_LS| / range(P_LS) <= 1e-4
    (P_LS the FP64 oracle's least-squares solution)."""
    from paper_2409_00184_b300.autograd import fit_gradient_descent
    N, n, p = 256, 32, 2
    field = synth.gm_noise_field(N, synth.BASE_SEED + 5, device="cuda")
    blocks = synth.blocks_from_field(field, n)
    ncp = synth.ncp_by_energy(synth.gradient_energy(blocks), (8, 12, 16), (100 / 3, 200 / 3))
    Dh = blocks.double().cpu().numpy()
    B = len(ncp)
    cps = [None] * B
    for C in (8, 12, 16):
        sel = np.nonzero(ncp == C)[0]
        kn = tuple(np.float32(synth.clamped_uniform_knots(C, p)).astype(np.float64) for _ in range(3))
        Pc = oenc.fit_separable_batch(Dh[sel], kn, (p, p, p))
        for m, b in enumerate(sel):
            cps[b] = Pc[m]
    bs = synth.make_block_set([(c, c, c) for c in ncp], [(p, p, p)] * B, [(n, n, n)] * B, cps)
    blk = mfa.DeviceBlocks(bs)
    P_ref = torch.from_numpy(np.concatenate([c.ravel() for c in cps])).cuda()
    D = blocks.contiguous().view(-1)
    P, hist = fit_gradient_descent(ctx, blk, D, n ** 3, B, iters=2000, tol=1e-4, P_ref=P_ref.float(),
                                   check_every=25, precision=mfa.PREC_SPLIT_BF16)
    assert ctx.device_status() == 0
    err = float((P.double() - P_ref).abs().max() / (P_ref.max() - P_ref.min()))
    print(f"split-BF16 GD: {hist[-1][0]} steps, {err:.2e}")
    assert err <= 1e-4, (err, hist[-5:])
