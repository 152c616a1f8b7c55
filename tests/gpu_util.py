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


# Knot vectors whose interior knots repeat (multiplicity up to p): spans jump over the empty intervals, so a
# sample's band can move by more than one control point from the previous sample's. (C, p, interior knots)
REPEATED_KNOT_AXES = [
    (8, 2, [1 / 4, 1 / 4, 1 / 2, 3 / 4, 3 / 4]),
    (10, 3, [1 / 4, 1 / 4, 1 / 2, 1 / 2, 1 / 2, 3 / 4]),
    (6, 1, [1 / 5, 2 / 5, 3 / 5, 4 / 5]),
    (12, 2, [1 / 8, 1 / 4, 1 / 4, 3 / 8, 1 / 2, 1 / 2, 5 / 8, 3 / 4, 7 / 8]),
    (7, 3, [3 / 8, 3 / 8, 5 / 8]),
]


def repeated_knot_set(nblocks, seed, nsamp_choices=(32,)):
    """Blocks whose three axes each take one of REPEATED_KNOT_AXES (seeded), control points U[-1, 1]."""
    g = synth.rng(seed)
    ncp, deg, ns, cps, kn = [], [], [], [], []
    for _ in range(nblocks):
        axes = [REPEATED_KNOT_AXES[int(i)] for i in g.integers(0, len(REPEATED_KNOT_AXES), 3)]
        ncp.append([a[0] for a in axes])
        deg.append([a[1] for a in axes])
        ns.append([int(g.choice(nsamp_choices)) for _ in range(3)])
        kn.append([np.array([0.0] * (p + 1) + list(t) + [1.0] * (p + 1)) for _, p, t in axes])
        cps.append(g.uniform(-1, 1, size=(ncp[-1][2], ncp[-1][1], ncp[-1][0])))
    return synth.make_block_set(ncp, deg, ns, cps, kn)
