"""Out-of-core rendering of micro-models (Sec. 4.3): caching (Algorithm 2), prefetching (Algorithm 3) and
rendering (Algorithm 4) per point of view.

Per frame: the previous frame's rendering is waited for and its prefetching stopped; the visible models
are looked up in the host LRU cache (misses are read from the store), packed and copied to the GPU in one
batch; the library decodes them into cache slots, the brick table maps each visible brick to its slot,
and the ray caster renders the frame. Then a background thread prefetches the models visible from the
predicted next point of view while the GPU renders. All of this is the library's native code (the store,
the cache and its thread, the kernels); this module only sequences the calls and builds the brick table.
"""

import time

import numpy as np
import torch

from . import mfa


def extrapolate_view(prev, cur):
    """Predicted next point of view: the eye moved again by its last displacement (target, frame and
    camera parameters kept)."""
    nxt = dict(cur)
    nxt["eye"] = tuple(2.0 * np.asarray(cur["eye"], dtype=np.float64) - np.asarray(prev["eye"], dtype=np.float64))
    return nxt


class OutOfCoreRenderer:
    """Renders frames of a brick grid whose micro-models live in a store file, through a host LRU cache
    of `capacity` models. brick_dims = (Bx, By, Bz); n = samples per brick axis; model b of the store is
    brick b (id = (bz*By + by)*Bx + bx). With `apron` the slots use the apron layout (mfa.DECODE_APRON): the
    decode is followed by the fill of the neighbour planes, and every ray-cast cell of a present brick reads
    its corners from one slot (the image is the same bit for bit)."""

    def __init__(self, ctx, store_path, capacity, brick_dims, n, tf, width, height, pinned=True, device="cuda",
                 apron=True):
        self.ctx, self.n, self.tf, self.apron = ctx, n, tf, apron
        self.stride = mfa.apron_voxels(n) if apron else n ** 3  # cache slot stride (voxels)
        self.B = tuple(int(b) for b in brick_dims)
        self.cache = mfa.ModelCache(store_path, capacity, pinned=pinned)
        count, max_ncp, max_degree = self.cache.info()
        if count != self.B[0] * self.B[1] * self.B[2]:
            raise ValueError("the store must hold one model per brick")
        self.batch = mfa.DeviceBatch(capacity, max_ncp, max_degree, device=device)
        self.slots = torch.empty(capacity * self.stride * 4, dtype=torch.float32, device=device)
        self.table_host = torch.full((self.B[2], self.B[1], self.B[0]), -1, dtype=torch.int32).pin_memory() \
            if pinned else torch.full((self.B[2], self.B[1], self.B[0]), -1, dtype=torch.int32)
        self.table = torch.full((self.B[2], self.B[1], self.B[0]), -1, dtype=torch.int32, device=device)
        self.image = torch.zeros(height, width, 4, dtype=torch.float32, device=device)
        self.width, self.height = width, height
        self.prefetching = False
        self.done = torch.cuda.Event()

    def frame(self, visible, view, predicted=None, stream=None):
        """Renders one frame of the visible brick ids; with `predicted` (the next view's visible ids),
        prefetches them while the frame renders. Returns the caching statistics of this frame."""
        stream = torch.cuda.current_stream() if stream is None else stream
        visible = np.ascontiguousarray(visible, dtype=np.int32)
        self.done.synchronize()  # the previous frame has rendered: its prefetching stops (Algorithm 3)
        pf = self.cache.prefetch_stop() if self.prefetching else {"loaded": 0, "bytes": 0}
        self.prefetching = False
        t0 = time.perf_counter_ns()
        look = self.cache.lookup(visible)
        self.cache.upload(visible, self.n, self.batch, stream=stream)
        self.table_host.fill_(-1)
        self.table_host.view(-1)[torch.from_numpy(visible.astype(np.int64))] = torch.arange(len(visible),
                                                                                            dtype=torch.int32)
        with torch.cuda.stream(stream):  # ordered before the fill and the ray cast that read it
            self.table.copy_(self.table_host, non_blocking=True)
        caching_ns = time.perf_counter_ns() - t0
        S, nv = self.stride, len(visible)
        mfa.decode_blocks(self.ctx, self.batch, self.slots, S, nv, bounds=self.batch.bounds,
                          flags=mfa.DECODE_APRON if self.apron else 0, stream=stream)
        if self.apron:
            mfa.fill_aprons(self.ctx, self.slots, S, nv, self.table, self.n, stream=stream)
        mfa.raycast(self.ctx, self.slots, S, nv, self.table, self.n, view, self.tf, self.image, stream=stream,
                    apron=self.apron)
        self.done.record(stream)
        if predicted is not None:
            self.cache.prefetch_start(np.ascontiguousarray(predicted, dtype=np.int32))
            self.prefetching = True
        return {"hits": look["hits"], "misses": look["misses"], "bytes_read": look["bytes"],
                "lookup_ns": look["ns"], "caching_ns": caching_ns, "prefetched": pf["loaded"],
                "prefetched_bytes": pf["bytes"]}

    def close(self):
        self.done.synchronize()
        if self.prefetching:
            self.cache.prefetch_stop()
        self.cache.close()
