"""Shared helpers for the GPU parity tests: workload builders (seeded inputs + oracle fits) and error metrics."""

import numpy as np
import torch

import synth
from oracle import decode, encode

# Tolerances relative to the field's value range (value) and to the largest gradient component
# (gradients), per precision; FP32 from the stated accuracy target of the FP32 decode.
TOL_FP32 = 1e-5


def rel_errors(got, want):
    """got/want: (..., 4) arrays of (f, f_u, f_v, f_w). Returns (value_err, [grad_err_u, v, w])."""
    got = np.asarray(got, dtype=np.float64).reshape(-1, 4)
    want = np.asarray(want, dtype=np.float64).reshape(-1, 4)
    vr = max(want[:, 0].max() - want[:, 0].min(), 1e-30)
    gmax = max(np.abs(want[:, 1:]).max(), 1e-30)
    ve = np.abs(got[:, 0] - want[:, 0]).max() / vr
    ge = [np.abs(got[:, c] - want[:, c]).max() / gmax for c in (1, 2, 3)]
    return ve, ge


def oracle_decode_set(bs, blocks=None):
    """Oracle decode of every (or the listed) block of a BlockSet: list of (n_z, n_y, n_x, 4)."""
    ids = range(len(bs)) if blocks is None else blocks
    return [decode.decode_block(bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b]) for b in ids]


def gm_blocks_fitted(N, n, C, p, seed, device="cpu"):
    """Gaussian-mixture + noise field on N^3 cut into n^3 bricks, each fitted by the oracle (C^3, degree p).

    Returns (BlockSet, field blocks as float32 numpy (B, n, n, n))."""
    field = synth.gm_noise_field(N, seed, device=device)
    blocks = synth.blocks_from_field(field, n).float().cpu().numpy()
    knots = tuple(synth.clamped_uniform_knots(C, p) for _ in range(3))
    # the oracle sees the FP32 knots the library reads
    k32 = tuple(np.float32(t).astype(np.float64) for t in knots)
    P = encode.fit_separable_batch(blocks, k32, (p, p, p))
    B = len(blocks)
    bs = synth.make_block_set([(C, C, C)] * B, [(p, p, p)] * B, [(n, n, n)] * B, list(P),
                              knots_list=[knots] * B)
    return bs, blocks


def oracle_fit_all(blocks, C, p, chunk=256):
    """Oracle least-squares control points (FP64) of every block of a (B, n, n, n) array, clamped uniform
    knots read in FP32 as the library reads them; chunked to bound host memory."""
    knots = tuple(np.float32(synth.clamped_uniform_knots(C, p)).astype(np.float64) for _ in range(3))
    out = [encode.fit_separable_batch(np.asarray(blocks[i:i + chunk], dtype=np.float64), knots, (p, p, p))
           for i in range(0, len(blocks), chunk)]
    return np.concatenate(out)


def node_groups(bs, slots_of=None):
    """Groups for oracle.raycast.decoded_nodes: the BlockSet's blocks grouped by (knots, degree, grid); the
    slot of block b is slots_of[b] (default: b)."""
    keys = {}
    for b in range(len(bs)):
        k = (tuple(bs.knot_off[b]), tuple(bs.degree[b]), tuple(bs.ncp[b]), tuple(bs.nsamp[b]))
        keys.setdefault(k, []).append(b)
    groups = []
    for k, ids in keys.items():
        Ps = np.stack([bs.block_cps(b) for b in ids])
        slots = np.asarray(ids if slots_of is None else [slots_of[b] for b in ids], dtype=np.int64)
        groups.append((slots, Ps, bs.block_knots(ids[0]), tuple(int(x) for x in k[1]), tuple(int(x) for x in k[3])))
    return groups



repeated_knot_set = synth.repeated_knot_set
