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


def mixed_blocks(ncps, degree, nsamp, device="cuda"):
    """DeviceBlocks of isotropic models with per-block NCP (ncps: int array), clamped uniform knots
    (one vector per distinct NCP), nsamp^3 samples; block b reads sample slot b."""
    ncps = np.asarray(ncps, dtype=np.int64)
    nb = len(ncps)
    vectors, offs, o = [], {}, 0
    for C in sorted(set(ncps.tolist())):
        t = clamped_uniform_knots(C, degree)
        offs[C] = o
        vectors.append(t)
        o += len(t)
    knots = np.concatenate(vectors) if vectors else np.zeros(0, np.float32)
    koff = np.array([offs[C] for C in ncps.tolist()], np.int64).reshape(-1, 1).repeat(3, axis=1)
    cp_off = np.concatenate([[0], np.cumsum(ncps ** 3)[:-1]]).astype(np.int64) if nb else np.zeros(0, np.int64)
    batch = _Batch(
        degree=np.full((nb, 3), degree, np.int32), ncp=np.repeat(ncps.reshape(-1, 1), 3, axis=1).astype(np.int32),
        nsamp=np.full((nb, 3), nsamp, np.int32), slot=np.arange(nb, dtype=np.int64), knot_off=koff,
        cp_off=cp_off, knots=knots)
    cps = torch.zeros(int((ncps ** 3).sum()), dtype=torch.float32, device=device)
    return mfa.DeviceBlocks(batch, device=device, cps=cps)


def cross_level_encode(ctx, field, n, degree, bound, levels, encode=True, search_all=False, stream=None):
    """Cross-level adaptive encoding (Sec. 4.2.3, Algorithm 1) of a float32 CUDA field (Nz, Ny, Nx).

    Level l (0 = finest) has micro-blocks of n^3 samples taken every 2^l samples. From the coarsest level
    to the finest: the blocks of the coarsest level, and at every finer level the blocks whose parent
    block is complex, are searched over NCP in [degree + 2, n] (Eq. 4 on the RMSE of each fit); a searched
    block is simple when its NCP* is degree + 2, complex otherwise (no candidate below the bound counts
    as complex and is encoded with NCP = n). Blocks that are not searched take NCP = degree + 1. The
    library fits at most MAX_NCP control points per axis, so for n > MAX_NCP the search stops there and a
    block with no candidate below the bound takes MAX_NCP.
    With `encode`, every level is then fitted with its per-block NCP in one batched call. With
    `search_all`, every block of every level is searched (in-level adaptive encoding alone, the baseline
    that Algorithm 1 speeds up).

    Returns a list, coarsest level first, of dicts: level, stride, blocks_per_axis, ncp (int32 numpy),
    searched, complex (bool numpy), fits (candidate fits run), and with `encode` blocks (DeviceBlocks
    holding the control points) and rmse (float64 CUDA tensor)."""
    Nz, Ny, Nx = field.shape
    cands = list(range(degree + 2, min(n, mfa.MAX_NCP) + 1))
    fallback = min(n, mfa.MAX_NCP)  # NCP of a block with no candidate below the bound
    out, parent_complex, parent_B = [], None, None
    for lvl in range(levels - 1, -1, -1):
        s = 2 ** lvl
        B = (Nx // (n * s), Ny // (n * s), Nz // (n * s))
        nb = B[0] * B[1] * B[2]
        if parent_complex is None or search_all:
            search = np.arange(nb)
        else:
            bz, by, bx = np.unravel_index(np.arange(nb), (B[2], B[1], B[0]))
            parent = ((bz // 2) * parent_B[1] + by // 2) * parent_B[0] + bx // 2
            search = np.nonzero(parent_complex[parent])[0]
        ncp = np.full(nb, degree + 1, np.int32)
        cplx = np.zeros(nb, bool)
        if len(search):
            ids = torch.as_tensor(search.astype(np.int32), device=field.device)
            D = mfa.lod_gather(ctx, field, n, s, ids=ids, stream=stream)
            sel, _ = search_ncp(ctx, D.view(-1), n, degree, bound, candidates=cands, keep_errors=False,
                                stream=stream)
            sel = sel.cpu().numpy()
            ncp[search] = np.where(sel > 0, sel, fallback)
            cplx[search] = sel != degree + 2
        rec = {"level": lvl, "stride": s, "blocks_per_axis": B, "ncp": ncp, "complex": cplx,
               "searched": np.isin(np.arange(nb), search), "fits": len(search) * len(cands)}
        if encode:
            D = mfa.lod_gather(ctx, field, n, s, stream=stream)
            blk = mixed_blocks(ncp, degree, n, device=field.device)
            plan = mfa.EncodePlan(ctx, blk)
            rmse = torch.empty(nb, dtype=torch.float64, device=field.device)
            mfa.encode_blocks(ctx, plan, D.view(-1), n ** 3, nb, blk.cps, rmse, stream=stream)
            plan.close()
            rec["blocks"], rec["rmse"] = blk, rmse
        out.append(rec)
        parent_complex, parent_B = cplx, B
    return out
