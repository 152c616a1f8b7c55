"""Out-of-core storage and caching (Algorithms 2 and 3) on the host, no GPU: the store's Eq. 2 layout, the
LRU cache against a reference LRU, and prefetching."""

import collections
import os
import time

import numpy as np
import pytest

import synth
from oracle import encode as oenc


@pytest.fixture(scope="module")
def mfa():
    from paper_2409_00184_b300 import mfa as m
    return m


def isotropic_blocks(count, seed):
    """Isotropic models (equal NCP and degree on the three axes), NCP in {3, 4, 6, 9}, degree 1..3."""
    g = synth.rng(seed)
    deg = g.integers(1, 4, count)
    ncp = np.maximum(g.choice([3, 4, 6, 9], count), deg + 1)
    cps = [g.uniform(-1, 1, (c, c, c)) for c in ncp]
    return synth.make_block_set([(c, c, c) for c in ncp], [(d, d, d) for d in deg], [(8, 8, 8)] * count, cps)


@pytest.fixture
def store(mfa, tmp_path):
    bs = isotropic_blocks(40, 1100)
    path = tmp_path / "models.mfa"
    mfa.store_write(path, bs)
    return path, bs


def test_store_layout_is_eq2(mfa, store):
    """Header (16 B) + index (16 B per model) + every model at exactly its Eq. 2 size."""
    path, bs = store
    sizes = [oenc.model_bytes(int(c), int(p)) for c, p in zip(bs.ncp[:, 0], bs.degree[:, 0])]
    assert os.path.getsize(path) == 16 + 16 * len(bs) + sum(sizes)
    raw = np.fromfile(path, dtype=np.uint8)
    assert bytes(raw[:8]) == b"MFAPACK1"
    idx = np.frombuffer(raw[16:16 + 16 * len(bs)].tobytes(), dtype=[("off", "<u8"), ("ncp", "<u4"), ("deg", "<u4")])
    for b in range(len(bs)):
        C, p, o = int(idx["ncp"][b]), int(idx["deg"][b]), int(idx["off"][b])
        assert (C, p) == (bs.ncp[b, 0], bs.degree[b, 0])
        assert raw[o] == p
        floats = np.frombuffer(raw[o + 1:o + sizes[b]].tobytes(), dtype="<f4")
        for a in range(3):  # the first C + p knots of each axis; the clamped last one is implied
            t = bs.knots[bs.knot_off[b, a]: bs.knot_off[b, a] + C + p]
            assert np.array_equal(floats[a * (C + p):(a + 1) * (C + p)], t)
        assert np.array_equal(floats[3 * (C + p):], bs.cps[bs.cp_off[b]: bs.cp_off[b] + C ** 3])


def test_store_rejects_anisotropic_models(mfa, tmp_path):
    bs = synth.random_block_set(4, 1101, ncp_choices=(3, 4, 6))
    bs.ncp[0] = (3, 4, 6)
    with pytest.raises(mfa.MfaError):
        mfa.store_write(tmp_path / "x.mfa", bs)


def test_lru_cache_matches_a_reference_lru(mfa, store):
    path, bs = store
    cache = mfa.ModelCache(path, capacity=12, pinned=False)
    assert cache.info() == (len(bs), int(bs.ncp.max()), int(bs.degree.max()))
    ref, g = collections.OrderedDict(), synth.rng(1102)
    sizes = [oenc.model_bytes(int(c), int(p)) for c, p in zip(bs.ncp[:, 0], bs.degree[:, 0])]
    for _ in range(60):
        ids = g.choice(len(bs), size=g.integers(1, 13), replace=False)
        hits = misses = nbytes = 0
        for i in ids:
            if i in ref:
                ref.move_to_end(i)
                hits += 1
            else:
                if len(ref) == 12:
                    ref.popitem(last=False)
                ref[i] = True
                misses += 1
                nbytes += sizes[i]
        st = cache.lookup(ids)
        assert (st["hits"], st["misses"], st["bytes"]) == (hits, misses, nbytes)
    with pytest.raises(mfa.MfaError):
        cache.lookup(np.arange(13))  # more than the capacity
    with pytest.raises(mfa.MfaError):
        cache.lookup([len(bs)])  # not in the store
    cache.close()


def test_prefetch_loads_the_predicted_models(mfa, store):
    path, bs = store
    cache = mfa.ModelCache(path, capacity=16, pinned=False)
    cache.lookup(np.arange(6))
    cache.prefetch_start(np.arange(3, 15))  # 3..5 are cached, 6..14 are not
    for _ in range(200):
        time.sleep(0.01)
        st = cache.prefetch_stop()
        if st["loaded"] == 9:
            break
        cache.prefetch_start(np.arange(3, 15))
    assert st["loaded"] == 9
    assert cache.lookup(np.arange(3, 15))["misses"] == 0
    with pytest.raises(mfa.MfaError):  # the cache is not used while a prefetch thread runs
        cache.prefetch_start([20])
        cache.lookup([0])
    cache.prefetch_stop()
    cache.close()
