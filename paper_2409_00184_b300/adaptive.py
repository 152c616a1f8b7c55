"""In-level adaptive encoding (Sec. 4.2.2, Eq. 4) on the library's kernels.

Every candidate NCP is fitted to every block of the batch by one batched least-squares encode
(mfa_encode_blocks: FP64 class set-up, FP32 fit, FP64 RMSE per block, Table 1's error metric),
and mfa_select_ncp then picks, per block, the smallest NCP whose RMSE is below the bound:
NCP* = argmin_NCP (Error(NCP) < e). The valid NCP range is [degree + 1, n]. All arithmetic runs in
the library; this module only builds descriptors and loops over the candidates.
"""

from types import SimpleNamespace

import numpy as np
import torch

from . import mfa


def clamped_uniform_knots(ncp, degree):
    """Clamped knot vector with uniform interior spans: degree+1 zeros, j/(ncp-degree), degree+1 ones."""
    inner = [j / (ncp - degree) for j in range(1, ncp - degree)]
    return np.array([0.0] * (degree + 1) + inner + [1.0] * (degree + 1), dtype=np.float32)


def uniform_blocks(nblocks, ncp, degree, nsamp, device="cuda"):
    """DeviceBlocks of `nblocks` isotropic models (ncp^3 control points, degree, nsamp^3 samples) that
    share one clamped uniform knot vector per axis; block b reads sample slot b."""
    t = clamped_uniform_knots(ncp, degree)
    L = len(t)
    batch = _Batch(
        degree=np.full((nblocks, 3), degree, np.int32), ncp=np.full((nblocks, 3), ncp, np.int32),
        nsamp=np.full((nblocks, 3), nsamp, np.int32), slot=np.arange(nblocks, dtype=np.int64),
        knot_off=np.tile(np.array([0, L, 2 * L], np.int64), (nblocks, 1)),
        cp_off=np.arange(nblocks, dtype=np.int64) * ncp ** 3, knots=np.concatenate([t, t, t]))
    cps = torch.zeros(nblocks * ncp ** 3, dtype=torch.float32, device=device)
    return mfa.DeviceBlocks(batch, device=device, cps=cps)


class _Batch(SimpleNamespace):
    """The per-block arrays DeviceBlocks reads, with the batch size as its length."""

    def __len__(self):
        return len(self.slot)


def candidate_ncps(degree, nsamp, max_ncp=mfa.MAX_NCP):
    """Every valid NCP of a block with nsamp samples per axis: degree + 1 .. min(nsamp, library maximum)."""
    return list(range(degree + 1, min(nsamp, max_ncp) + 1))


def search_ncp(ctx, data, nsamp, degree, bound, candidates=None, keep_errors=True, stream=None):
    """Eq. 4 for every block of `data` (float32 CUDA tensor, block b's nsamp^3 samples at b*nsamp^3).

    Returns (ncp_star, errors): ncp_star int32 (B,) with -1 where no candidate meets the bound;
    errors float64 (len(candidates), B), the RMSE of every candidate fit."""
    candidates = candidate_ncps(degree, nsamp) if candidates is None else list(candidates)
    vox = nsamp ** 3
    B = data.numel() // vox
    errors = torch.empty((len(candidates), B), dtype=torch.float64, device=data.device)
    cps = None
    for c, C in enumerate(candidates):
        blk = uniform_blocks(B, C, degree, nsamp, device=data.device)
        if cps is None or cps.numel() < blk.cps_len:
            cps = torch.empty(blk.cps_len, dtype=torch.float32, device=data.device)
        plan = mfa.EncodePlan(ctx, blk)
        mfa.encode_blocks(ctx, plan, data, vox, B, cps, errors[c], stream=stream)
        plan.close()
    ncp = mfa.select_ncp(ctx, errors, candidates, bound, stream=stream)
    return ncp, (errors if keep_errors else None)
