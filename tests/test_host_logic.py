"""Host-side logic of the package that needs no GPU: the autotuner's batch-class key and its JSON round
trip, the NCP candidates of Eq. 4's search, the clamped uniform knot vector, and the next point of view
that the out-of-core prefetcher (Algorithm 3) predicts."""

import numpy as np

import synth


class _FakeCtx:
    """Records the decode tilings a loader installs (the library call is not made)."""

    def __init__(self):
        self.installed = {}

    def set_decode_tiling(self, bounds, ks, ctas):
        self.installed[(bounds.max_degree, bounds.max_ncp, bounds.max_nsamp)] = (ks, ctas)


def test_autotune_key_and_json_round_trip(tmp_path):
    from paper_2409_00184_b300 import autotune, mfa
    assert autotune.key_of(mfa.Bounds(2, 24, 32)) == "p2_C24_n32"
    results = [{"key": "p2_C24_n32", "ks": 2, "ctas_per_sm": 0, "us": 919.2},
               {"key": "p3_C12_n64", "ks": 8, "ctas_per_sm": 4, "us": 101.5}]
    path = tmp_path / "tuning.json"
    autotune.save(path, results)
    ctx = _FakeCtx()
    data = autotune.load(path, ctx)
    assert ctx.installed == {(2, 24, 32): (2, 0), (3, 12, 64): (8, 4)}
    assert data["p3_C12_n64"]["us"] == 101.5


def test_candidate_ncps_span_degree_plus_one_to_n():
    """Sec. 4.2.2: every NCP from degree + 1 up to the block's sample count (and the library's maximum)."""
    from paper_2409_00184_b300 import adaptive, mfa
    assert adaptive.candidate_ncps(2, 8) == [3, 4, 5, 6, 7, 8]
    assert adaptive.candidate_ncps(3, 64) == list(range(4, mfa.MAX_NCP + 1))
    assert adaptive.candidate_ncps(1, 2) == [2]


def test_clamped_uniform_knots_match_the_generator():
    """The package's knot vector (FP32, as the library reads it) is the seeded inputs' clamped uniform one."""
    from paper_2409_00184_b300 import adaptive
    for C, p in ((3, 2), (12, 2), (24, 3), (5, 1)):
        t = adaptive.clamped_uniform_knots(C, p)
        assert t.dtype == np.float32 and len(t) == C + p + 1
        assert np.array_equal(t, synth.clamped_uniform_knots(C, p).astype(np.float32))
        assert np.all(t[:p + 1] == 0) and np.all(t[-(p + 1):] == 1) and np.all(np.diff(t) >= 0)


def test_next_view_repeats_the_last_displacement():
    from paper_2409_00184_b300 import outofcore
    prev = synth.orbit_view(3)
    cur = synth.orbit_view(4)
    nxt = outofcore.extrapolate_view(prev, cur)
    want = 2 * np.asarray(cur["eye"]) - np.asarray(prev["eye"])
    assert np.allclose(nxt["eye"], want, rtol=0, atol=1e-12)
    assert nxt["target"] == cur["target"] and nxt["fov_y_deg"] == cur["fov_y_deg"]
    assert cur["eye"] == synth.orbit_view(4)["eye"]  # the current view is left as it was
