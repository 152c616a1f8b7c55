"""Differentiable least-squares encode on top of the library's decode and adjoint kernels.

`DecodeValue` is a torch.autograd.Function: forward = value-only decode of every block's control
points (mfa_decode_blocks, MFA_DECODE_VALUE_ONLY), backward = the transposed contraction of the
incoming gradient (mfa_adjoint_blocks). The basis is recomputed from the knots inside both kernels;
nothing but the control points is saved for backward.

`fit_gradient_descent` fits control points to sample grids by (Nesterov-accelerated) gradient
descent on 0.5*||decode(P) - D||^2 (the least-squares fit of Algorithm 1's model()), using the
library's fused gradient kernel (N^T N P - N^T D) and a per-block step 1/L, with L the largest
eigenvalue of that block's Gram operator (found by power iteration through the same kernel). With
precision BF16 or split-BF16 the gradient is the FP32 residual decode (mfa_decode_compare_blocks) followed
by the tensor-core adjoint in that precision (mfa_adjoint_blocks), and L comes from the same two calls.
The arithmetic of every decode, adjoint and gradient runs in the library; the optimizer's vector
updates are torch tensor operations.
"""

import torch

from . import mfa


class DecodeValue(torch.autograd.Function):
    """f = decode_value(P) on each block's sample grid (slot-addressed, slot_stride floats per slot). The
    forward decode and the backward adjoint run in `precision` (FP32 on the CUDA cores, or BF16 /
    split-BF16 on the tensor cores, where the adjoint takes 32 samples and at most 16 control points)."""

    @staticmethod
    def forward(fctx, cps, lib_ctx, blocks, slot_stride, nslots, precision=mfa.PREC_FP32):
        out = torch.zeros(nslots * slot_stride, device=cps.device, dtype=torch.float32)
        mfa.decode_blocks(lib_ctx, blocks, out, slot_stride, nslots, flags=mfa.DECODE_VALUE_ONLY,
                          cps=cps.contiguous(), precision=precision)
        fctx.lib = (lib_ctx, blocks, slot_stride, nslots, precision)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        lib_ctx, blocks, slot_stride, nslots, precision = fctx.lib
        grad = torch.empty(blocks.cps_len, device=grad_out.device, dtype=torch.float32)
        mfa.adjoint_blocks(lib_ctx, blocks, grad_out.contiguous(), slot_stride, nslots, grad, precision=precision)
        return grad, None, None, None, None, None


def decode_value(cps, lib_ctx, blocks, slot_stride, nslots, precision=mfa.PREC_FP32):
    return DecodeValue.apply(cps, lib_ctx, blocks, slot_stride, nslots, precision)


def block_ids(blocks, device="cuda"):
    """Block index of every control point (for per-block reductions)."""
    sizes = torch.as_tensor((blocks.host_desc["ncp"].astype("int64")).prod(axis=1), device=device)
    return torch.repeat_interleave(torch.arange(blocks.n, device=device), sizes)


class Gradient:
    """G = N^T (decode(P) - D) per block: the fused FP32 kernel, or (BF16 / split-BF16) the FP32 residual
    decode followed by the tensor-core adjoint in that precision."""

    def __init__(self, lib_ctx, blocks, slot_stride, nslots, precision=mfa.PREC_FP32):
        self.args = (lib_ctx, blocks, slot_stride, nslots)
        self.precision = precision
        if precision != mfa.PREC_FP32:
            dev = blocks.cps.device
            self.f = torch.empty(nslots * slot_stride, device=dev)
            self.R = torch.empty(nslots * slot_stride, device=dev)

    def __call__(self, P, data, G):
        lib_ctx, blocks, slot_stride, nslots = self.args
        if self.precision == mfa.PREC_FP32:
            mfa.adjoint_blocks(lib_ctx, blocks, data, slot_stride, nslots, G, cps=P)
        else:
            mfa.decode_compare_blocks(lib_ctx, blocks, self.f, slot_stride, nslots, data, slot_stride, residual=self.R,
                                      flags=mfa.DECODE_VALUE_ONLY, cps=P)
            mfa.adjoint_blocks(lib_ctx, blocks, self.R, slot_stride, nslots, G, precision=self.precision)


def lipschitz(lib_ctx, blocks, slot_stride, nslots, iters=30, seed=0, precision=mfa.PREC_FP32):
    """Per-block largest eigenvalue of N^T N (the gradient's Lipschitz constant), by power iteration
    with the gradient at zero data: G(P; D = 0) = N^T N P."""
    dev = blocks.cps.device
    ids = block_ids(blocks, dev)
    zero = torch.zeros(nslots * slot_stride, device=dev)
    grad = Gradient(lib_ctx, blocks, slot_stride, nslots, precision)
    g = torch.Generator(device=dev).manual_seed(seed)
    v = torch.rand(blocks.cps_len, device=dev, generator=g) + 0.5
    lam = torch.zeros(blocks.n, device=dev)
    hv = torch.empty_like(v)
    for _ in range(iters):
        nrm = torch.zeros(blocks.n, device=dev).index_add_(0, ids, v * v).sqrt()
        v = v / nrm[ids]
        grad(v, zero, hv)
        lam = torch.zeros(blocks.n, device=dev).index_add_(0, ids, v * hv)
        v = hv.clone()
    return lam


def fit_gradient_descent(lib_ctx, blocks, data, slot_stride, nslots, iters=2000, nesterov=True, P0=None,
                         tol=None, P_ref=None, check_every=25, precision=mfa.PREC_FP32):
    """Least-squares control points by gradient descent with per-block step 1/L, the gradient in FP32 or (the
    adjoint on the tensor cores) BF16 / split-BF16.

    Stops after `iters` steps or, with P_ref given, once max|P - P_ref| / range(P_ref) <= tol (checked
    every `check_every` steps). Returns (P, history of (step, relative error))."""
    dev = blocks.cps.device
    ids = block_ids(blocks, dev)
    grad = Gradient(lib_ctx, blocks, slot_stride, nslots, precision)
    L = lipschitz(lib_ctx, blocks, slot_stride, nslots, precision=precision) * 1.01
    step = (1.0 / L)[ids]
    P = torch.zeros(blocks.cps_len, device=dev) if P0 is None else P0.clone()
    Y, P_prev = P.clone(), P.clone()
    G = torch.empty_like(P)
    hist = []
    rng = None if P_ref is None else float(P_ref.max() - P_ref.min())
    for k in range(1, iters + 1):
        grad(Y if nesterov else P, data, G)
        P_new = (Y if nesterov else P) - step * G
        if nesterov:
            Y = P_new + (k - 1.0) / (k + 2.0) * (P_new - P_prev)
            P_prev = P_new
        P = P_new
        if P_ref is not None and (k % check_every == 0 or k == iters):
            err = float((P - P_ref).abs().max()) / rng
            hist.append((k, err))
            if tol is not None and err <= tol:
                break
    return P, hist
