"""Autotuner for the decode's tile shape (z-planes per work unit, resident CTAs per SM).

For a batch class - the (max_degree, max_ncp, max_nsamp) bounds of a decode call - it times
candidate tilings of mfa_decode_blocks with CUDA events on the calling stream and stores the
fastest in the context (mfa_ctx_set_decode_tiling); results can be saved to and loaded from JSON
keyed by the class. Timing is host orchestration only: every timed call runs the library's kernel.
"""

import json

import torch

from . import mfa

DEFAULT_KS = (2, 4, 8, 16)
DEFAULT_CTAS = (0, 2, 3, 4, 6)


def key_of(bounds):
    return f"p{bounds.max_degree}_C{bounds.max_ncp}_n{bounds.max_nsamp}"


def tune_decode(ctx, blocks, cache, slot_stride, nslots, ks_candidates=DEFAULT_KS, cta_candidates=DEFAULT_CTAS,
                iters=10, warmup=2, list_=None, count=None, flags=0):
    """Times every (ks, ctas_per_sm) pair on this batch; installs and returns the fastest.

    Returns {"key": ..., "ks": ..., "ctas_per_sm": ..., "us": ..., "table": [(ks, ctas, us), ...]}."""
    b = blocks.bounds
    table = []
    stream = torch.cuda.current_stream()
    for ks in ks_candidates:
        if ks > b.max_nsamp:
            continue
        for ctas in cta_candidates:
            ctx.set_decode_tiling(b, ks, ctas)
            for _ in range(warmup):
                mfa.decode_blocks(ctx, blocks, cache, slot_stride, nslots, flags=flags, list_=list_, count=count)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(iters):
                mfa.decode_blocks(ctx, blocks, cache, slot_stride, nslots, flags=flags, list_=list_, count=count)
            e1.record(stream)
            e1.synchronize()
            table.append((ks, ctas, e0.elapsed_time(e1) / iters * 1e3))
    ks, ctas, us = min(table, key=lambda r: r[2])
    ctx.set_decode_tiling(b, ks, ctas)
    return {"key": key_of(b), "ks": ks, "ctas_per_sm": ctas, "us": us, "table": table}


def save(path, results):
    with open(path, "w") as f:
        json.dump({r["key"]: {"ks": r["ks"], "ctas_per_sm": r["ctas_per_sm"], "us": r["us"]} for r in results},
                  f, indent=1)


def load(path, ctx):
    """Installs every entry of a saved tuning file into the context."""
    with open(path) as f:
        data = json.load(f)
    for key, v in data.items():
        p, C, n = (int(t[1:]) for t in key.split("_"))
        ctx.set_decode_tiling(mfa.Bounds(p, C, n), v["ks"], v["ctas_per_sm"])
    return data
