"""Differentiable least-squares encode: DecodeValue (torch.autograd.Function over the decode and the
adjoint kernel) and gradient-descent fitting against the FP64 oracle's least-squares solve."""

import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj
from oracle import decode as odec
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


def test_autograd_gradient_matches_finite_differences_and_oracle(mfa, ctx):
    """4^3 control points, 8^3 samples: autograd gradient of 0.5*||decode(P) - D||^2 vs central FD and vs the
    oracle's adjoint of the oracle's residual."""
    from paper_2409_00184_b300.autograd import decode_value
    bs = synth.random_block_set(6, 501, ncp_choices=(4,), nsamp_choices=(8,), degree_choices=(2, 3),
                                anisotropic=False)
    blk = mfa.DeviceBlocks(bs)
    g = synth.rng(501)
    D = torch.from_numpy(g.uniform(-1, 1, (len(bs), 512)).astype(np.float32).ravel()).cuda()
    P = blk.cps.clone().requires_grad_(True)
    f = decode_value(P, ctx, blk, 512, len(bs))
    loss = 0.5 * ((f.double() - D.double()) ** 2).sum()
    loss.backward()
    grad = P.grad.cpu().numpy()
    assert ctx.device_status() == 0

    def L(Pt):
        with torch.no_grad():
            ff = decode_value(Pt, ctx, blk, 512, len(bs))
            return 0.5 * float(((ff.double() - D.double()) ** 2).sum())

    h = 0.05
    for idx in g.choice(blk.cps_len, 24, replace=False):
        e = torch.zeros_like(blk.cps)
        e[idx] = h
        fd = (L(blk.cps + e) - L(blk.cps - e)) / (2 * h)  # exact for a quadratic, up to FP32 rounding
        assert abs(fd - grad[idx]) <= 2e-3 * max(1.0, np.abs(grad).max()), (idx, fd, grad[idx])
    Dn = D.cpu().numpy().reshape(len(bs), 8, 8, 8).astype(np.float64)
    for b in range(len(bs)):
        kn, deg = bs.block_knots(b), bs.degree[b]
        r = odec.decode_block(bs.block_cps(b), kn, deg, bs.nsamp[b])[..., 0] - Dn[b]
        want = oadj.adjoint_block(r, kn, deg, bs.ncp[b])
        got = grad[bs.cp_off[b]: bs.cp_off[b] + 64].reshape(4, 4, 4)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_fused_gradient_equals_autograd(mfa, ctx):
    """The fused gradient kernel (adjoint with control points) equals decode-then-adjoint through autograd."""
    from paper_2409_00184_b300.autograd import decode_value
    bs = synth.random_block_set(16, 502, ncp_choices=(6, 8, 12), nsamp_choices=(32,), degree_choices=(2,))
    blk = mfa.DeviceBlocks(bs)
    D = torch.rand(len(bs) * 32 ** 3, device="cuda")
    P = blk.cps.clone().requires_grad_(True)
    f = decode_value(P, ctx, blk, 32 ** 3, len(bs))
    (0.5 * ((f - D) ** 2).sum()).backward()
    G = torch.empty(blk.cps_len, device="cuda")
    mfa.adjoint_blocks(ctx, blk, D, 32 ** 3, len(bs), G, cps=blk.cps)
    assert ctx.device_status() == 0
    assert float((G - P.grad).abs().max()) <= 1e-5 * float(P.grad.abs().max())


@pytest.mark.parametrize("name", ["split", "bf16"])
def test_autograd_tensor_core_precisions(mfa, ctx, name):
    """decode_value with a tensor-core precision: the forward value-only decode and the backward adjoint both
    on the tensor cores, against the oracle's decode and the oracle's adjoint of the oracle's residual.
    Tolerances: the value as the decode's (split-BF16 1e-4, BF16 1e-2 of the value range); the gradient as
    the sum of the decode's and the adjoint's (the residual carries the decode's error into the adjoint)."""
    from paper_2409_00184_b300.autograd import decode_value
    prec, tol = {"split": (mfa.PREC_SPLIT_BF16, 1e-4), "bf16": (mfa.PREC_BF16, 1e-2)}[name]
    bs = synth.random_block_set(12, 503, ncp_choices=(6, 8, 12), nsamp_choices=(32,), degree_choices=(2, 3))
    blk = mfa.DeviceBlocks(bs)
    g = synth.rng(503)
    D = torch.from_numpy(g.uniform(-1, 1, (len(bs), 32 ** 3)).astype(np.float32).ravel()).cuda()
    P = blk.cps.clone().requires_grad_(True)
    f = decode_value(P, ctx, blk, 32 ** 3, len(bs), precision=prec)
    (0.5 * ((f - D) ** 2).sum()).backward()
    assert ctx.device_status() == 0
    fh, grad = f.detach().cpu().numpy().reshape(len(bs), -1), P.grad.cpu().numpy()
    Dn = D.cpu().numpy().reshape(len(bs), 32, 32, 32).astype(np.float64)
    vmax, gmax = 0.0, 0.0
    for b in range(len(bs)):
        kn, deg = bs.block_knots(b), bs.degree[b]
        fo = odec.decode_block(bs.block_cps(b), kn, deg, bs.nsamp[b])[..., 0]
        vmax = max(vmax, np.abs(fh[bs.slot[b]].reshape(32, 32, 32) - fo).max() / (fo.max() - fo.min()))
        want = oadj.adjoint_block(fo - Dn[bs.slot[b]], kn, deg, bs.ncp[b])
        Cx, Cy, Cz = bs.ncp[b]
        got = grad[bs.cp_off[b]: bs.cp_off[b] + Cx * Cy * Cz].reshape(Cz, Cy, Cx)
        gmax = max(gmax, np.abs(got - want).max() / np.abs(want).max())
    print(f"{name} autograd: value {vmax:.2e}, gradient {gmax:.2e}")
    assert vmax <= tol and gmax <= 2 * tol, (vmax, gmax)


def test_gradient_descent_fit_256cubed_512_blocks(mfa, ctx):
    """256^3 Gaussian-mixture+noise field, 512 blocks of 32^3, degree 2, C in {8, 12, 16} by gradient-energy
    terciles; Nesterov gradient descent with per-block step 1/L until max|P - P_LS| / range(P_LS) <= 1e-5,
    P_LS the FP64 oracle's least-squares solution, within 2000 steps."""
    from paper_2409_00184_b300.autograd import fit_gradient_descent
    N, n, p = 256, 32, 2
    field = synth.gm_noise_field(N, synth.BASE_SEED + 5, device="cuda")
    blocks = synth.blocks_from_field(field, n)
    ncp = synth.ncp_by_energy(synth.gradient_energy(blocks), (8, 12, 16), (100 / 3, 200 / 3))
    Dh = blocks.double().cpu().numpy()
    B = len(ncp)
    cps = [None] * B
    for C in (8, 12, 16):  # FP64 normal-equation solve per class (the library reads FP32 knots)
        sel = np.nonzero(ncp == C)[0]
        kn = tuple(np.float32(synth.clamped_uniform_knots(C, p)).astype(np.float64) for _ in range(3))
        Pc = oenc.fit_separable_batch(Dh[sel], kn, (p, p, p))
        for m, b in enumerate(sel):
            cps[b] = Pc[m]
    bs = synth.make_block_set([(c, c, c) for c in ncp], [(p, p, p)] * B, [(n, n, n)] * B, cps)
    blk = mfa.DeviceBlocks(bs)
    P_ref = torch.from_numpy(np.concatenate([c.ravel() for c in cps])).cuda()
    D = blocks.contiguous().view(-1)
    P, hist = fit_gradient_descent(ctx, blk, D, n ** 3, B, iters=2000, tol=1e-5, P_ref=P_ref.float(),
                                   check_every=25)
    assert ctx.device_status() == 0
    err = float((P.double() - P_ref).abs().max() / (P_ref.max() - P_ref.min()))
    assert err <= 1e-5, (err, hist[-5:])
    assert hist[-1][0] <= 2000
