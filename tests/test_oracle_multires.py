"""Pins for the oracle's multi-resolution partition, LOD selection, LOD rendering and image metrics."""

import math

import numpy as np
import pytest

import synth
from oracle import encode, multires, raycast


def _field(N, seed):
    return synth.rng(seed).uniform(-1, 1, (N, N + 4, N + 8))


def test_shared_blocks_share_their_boundary_samples():
    n, s = 5, 2
    F = _field(2 * (n - 1) * s + 1, 61)[:, :2 * (n - 1) * s + 1, :3 * (n - 1) * s + 1]
    blocks, (Bx, By, Bz) = multires.shared_blocks(F, n, s)
    assert (Bx, By, Bz) == (3, 2, 2) and blocks.shape == (12, n, n, n)
    bid = lambda x, y, z: (z * By + y) * Bx + x  # noqa: E731
    for z in range(Bz):
        for y in range(By):
            for x in range(Bx - 1):
                assert np.array_equal(blocks[bid(x, y, z)][:, :, -1], blocks[bid(x + 1, y, z)][:, :, 0])
    assert np.array_equal(blocks[bid(0, 0, 0)][:, -1, :], blocks[bid(0, 1, 0)][:, 0, :])
    assert np.array_equal(blocks[bid(1, 0, 0)][-1, :, :], blocks[bid(1, 0, 1)][0, :, :])
    # element by element against the node each sample stands for
    b = bid(2, 1, 1)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                assert blocks[b][k, j, i] == F[(n - 1) * s + k * s, (n - 1) * s + j * s, 2 * (n - 1) * s + i * s]
    whole, B = multires.shared_blocks(F[:9, :9, :9], 9, 1)
    assert B == (1, 1, 1) and np.array_equal(whole[0], F[:9, :9, :9])
    with pytest.raises(ValueError):
        multires.shared_blocks(F[:10, :9, :9], 9, 1)


def _level_rule(eye, B0, n, levels, ranges):
    """The selection per finest block without the recursion: the coarsest ancestor level l >= 1 whose block is
    far enough, else level 0 (the top-down walk stops at the first far-enough ancestor)."""
    off, _ = multires.level_offsets(B0, levels)
    N = B0 * (n - 1) + 1
    out = np.zeros((B0, B0, B0), dtype=np.int64)
    for z in range(B0):
        for y in range(B0):
            for x in range(B0):
                chosen = 0
                for lvl in range(levels - 1, 0, -1):
                    E = (n - 1) << lvl
                    ax, ay, az = x >> lvl, y >> lvl, z >> lvl
                    if multires._far_enough((ax * E, ay * E, az * E), E, N, eye, ranges[lvl - 1]):
                        chosen = lvl
                        break
                Bl = B0 >> chosen
                out[z, y, x] = off[chosen] + ((z >> chosen) * Bl + (y >> chosen)) * Bl + (x >> chosen)
    return out


@pytest.mark.parametrize("eye", [(0.1, 0.2, -0.3), (1.3, -0.4, 0.9), (-1.6, 1.0, 0.5)])
def test_lod_selection_top_down_equals_the_per_block_rule(eye):
    B0, n, levels = 8, 5, 4
    t = multires.select_lod(eye, B0, n, levels)
    assert np.array_equal(t, _level_rule(eye, B0, n, levels, multires.DEFAULT_RANGES))
    lv = np.array([[[multires.block_geometry(int(b), B0, n, levels)[0] for b in row] for row in pl] for pl in t])
    assert len(np.unique(lv)) >= 2  # these views mix levels


def test_lod_selection_closed_cases():
    B0, n, levels = 8, 5, 4
    off, total = multires.level_offsets(B0, levels)
    assert off == [0, 512, 576, 584] and total == 585
    far = multires.select_lod((40.0, 0.0, 0.0), B0, n, levels)
    assert np.all(far == 584)  # the whole volume from the single coarsest block
    near = multires.select_lod((0.0, 0.0, 0.0), B0, n, levels, ranges=(10.0, 20.0, 30.0))
    assert np.array_equal(near.ravel(), np.arange(512))  # every finest block itself
    # the distance ranges hold for what is selected: a block of level l >= 1 is at least ranges[l-1] away,
    # and the parent of a block below the coarsest level is nearer than the parent's range
    eye = (0.9, 0.1, -0.2)
    t = multires.select_lod(eye, B0, n, levels)
    N = B0 * (n - 1) + 1
    for bid in np.unique(t):
        lvl, g0, E = multires.block_geometry(int(bid), B0, n, levels)
        c = np.array([(2 * g0[a] + E) / (N - 1) - 1 for a in range(3)])
        d = np.linalg.norm(c - np.array(eye))
        if lvl >= 1:
            assert d >= multires.DEFAULT_RANGES[lvl - 1] - 1e-6
        if lvl < levels - 1:
            Ep = 2 * E
            gp = [g // Ep * Ep for g in g0]
            cp = np.array([(2 * gp[a] + Ep) / (N - 1) - 1 for a in range(3)])
            assert np.linalg.norm(cp - np.array(eye)) < multires.DEFAULT_RANGES[lvl] + 1e-6


def _poly(g):
    x, y, z = g[:, 0], g[:, 1], g[:, 2]
    f = 0.3 + 0.02 * x - 0.01 * y + 0.015 * z + 1e-3 * x * y - 2e-3 * z * z + 5e-4 * x * z
    grad = np.stack([0.02 + 1e-3 * y + 5e-4 * z, -0.01 + 1e-3 * x, 0.015 - 4e-3 * z + 5e-4 * x], axis=1)
    return f, grad


def _poly_models(B0, n, levels, p=2, C=4):
    """Every block of every level fitted (least squares, exact for a polynomial of degree <= p per axis) to
    the quadratic field _poly over its own nodes."""
    off, total = multires.level_offsets(B0, levels)
    knots = tuple(synth.clamped_uniform_knots(C, p) for _ in range(3))
    models = {}
    for bid in range(total):
        _, g0, E = multires.block_geometry(bid, B0, n, levels)
        s = np.arange(n) * (E / (n - 1))
        Z, Y, X = np.meshgrid(g0[2] + s, g0[1] + s, g0[0] + s, indexing="ij")
        D = _poly(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1))[0].reshape(n, n, n)
        models[bid] = (encode.fit_separable(D, knots, (p, p, p)), knots, (p, p, p))
    return lambda b: models[b]


def test_fetch_lod_reproduces_a_global_polynomial_at_any_selection():
    """Models that reproduce one quadratic field give that field and its node-unit gradient wherever a sample
    falls, whatever level the selection chose there (checks the block lookup, u, and the gradient scale)."""
    B0, n, levels = 4, 5, 3
    models = _poly_models(B0, n, levels)
    g = synth.rng(62).uniform(0, B0 * (n - 1), (400, 3))
    for eye in ((0.0, 0.0, 0.0), (1.7, 0.2, -0.1), (9.0, 9.0, 9.0)):
        t = multires.select_lod(eye, B0, n, levels, ranges=(0.8, 1.6))
        got = multires.fetch_lod(models, t, n, levels, g)
        f, grad = _poly(g)
        assert np.max(np.abs(got[:, 0] - f)) < 1e-12
        assert np.max(np.abs(got[:, 1:] - grad)) < 1e-12


def test_raycast_lod_equals_the_cache_render_of_a_linear_field():
    """For a linear field the trilinear cache render is exact, and so are the selected models: the LOD render
    (shared-boundary nodes, N = B0 (n-1) + 1) equals the cache renderer's image over one brick of N^3 nodes."""
    B0, n, levels = 4, 5, 3
    N = B0 * (n - 1) + 1
    a = np.array([0.012, -0.008, 0.01])

    def lin(g):
        return 0.5 + g @ a

    off, total = multires.level_offsets(B0, levels)
    knots = tuple(synth.clamped_uniform_knots(2, 1) for _ in range(3))
    models = {}
    for bid in range(total):
        _, g0, E = multires.block_geometry(bid, B0, n, levels)
        P = np.zeros((2, 2, 2))
        for c in (0, 1):
            for b in (0, 1):
                for d in (0, 1):
                    P[c, b, d] = lin(np.array([g0[0] + d * E, g0[1] + b * E, g0[2] + c * E], dtype=float))
        models[bid] = (P, knots, (1, 1, 1))
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    cache = np.zeros((1, N, N, N, 4))
    cache[0, ..., 0] = 0.5 + a[0] * i + a[1] * j + a[2] * k
    cache[0, ..., 1:] = a * (N - 1)  # parametric gradient of the single brick (u = g / (N - 1))
    tf = synth.transfer_function(7)
    view = synth.default_view(width=21, height=17, opacity_max=0.97)
    want = raycast.raycast(cache, np.zeros((1, 1, 1), np.int32), N, view, tf)
    for eye in ((0.4, 0.1, 0.2), (2.2, 1.6, 2.0)):
        t = multires.select_lod(eye, B0, n, levels, ranges=(0.8, 1.6))
        got = multires.raycast_lod(lambda b: models[b], t, n, levels, view, tf)
        assert np.max(np.abs(got - want)) < 1e-12
    assert (want[..., 3] > 0).mean() > 0.5


def test_mse_and_psnr_closed_forms():
    a = synth.rng(63).uniform(0, 1, (9, 7, 4))
    assert multires.mse(a, a) == 0.0 and multires.psnr(a, a) == math.inf
    assert abs(multires.mse(a, a + 0.05) - 0.0025) < 1e-15
    assert abs(multires.psnr(a, a + 0.05) - 20 * math.log10(1 / 0.05)) < 1e-10  # 26.0206 dB
    b = a.copy()
    b[0, 0, 0] += 0.6  # one channel of one pixel off by 0.6: MSE = 0.36 / 252
    assert abs(multires.mse(a, b) - 0.36 / 252) < 1e-15
    assert abs(multires.psnr(a, b, peak=2.0) - 10 * math.log10(4 * 252 / 0.36)) < 1e-10


def _ssim_brute(a, b, size=11, sigma=1.5, c1=1e-4, c2=9e-4):
    """SSIM of one channel with every window's weighted statistics summed directly (no separable filter)."""
    x = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-0.5 * (x / sigma) ** 2)
    w2 = np.outer(g, g) / np.outer(g, g).sum()
    H, W = a.shape
    vals = []
    for i in range(H - size + 1):
        for j in range(W - size + 1):
            pa, pb = a[i:i + size, j:j + size], b[i:i + size, j:j + size]
            ma, mb = (w2 * pa).sum(), (w2 * pb).sum()
            va = (w2 * (pa - ma) ** 2).sum()
            vb = (w2 * (pb - mb) ** 2).sum()
            cab = (w2 * (pa - ma) * (pb - mb)).sum()
            vals.append(((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2)))
    return np.mean(vals)


def test_ssim_against_per_window_sums_and_closed_forms():
    """SSIM (Sec. 5.2): equal to the per-window weighted sums written out, 1 for equal images, symmetric, the
    closed form (2 c c' + c1) / (c^2 + c'^2 + c1) for two constant images, and below 1 for a noisy copy."""
    g = synth.rng(64)
    a = g.uniform(0, 1, (17, 19))
    b = np.clip(a + g.normal(0, 0.05, a.shape), 0, 1)
    assert abs(multires.ssim(a, b) - _ssim_brute(a, b)) < 1e-12
    assert abs(multires.ssim(a, a) - 1.0) < 1e-12
    assert abs(multires.ssim(a, b) - multires.ssim(b, a)) < 1e-12
    assert multires.ssim(a, b) < 0.99
    c, d = 0.3, 0.7
    want = (2 * c * d + 1e-4) / (c * c + d * d + 1e-4)
    assert abs(multires.ssim(np.full((15, 15), c), np.full((15, 15), d)) - want) < 1e-12
    rgba = g.uniform(0, 1, (16, 14, 4))
    per = [multires.ssim(rgba[..., k], rgba[..., k] * 0.9) for k in range(4)]
    assert abs(multires.ssim(rgba, rgba * 0.9) - np.mean(per)) < 1e-12


def test_ssim_gaussian_window():
    """The structural-similarity window: symmetric, normalised, peaked at the centre, with the variance of
    the sampled Gaussian (sigma^2 = 2.25 up to the truncation at +-5 taps)."""
    w = multires.gaussian_window()
    x = np.arange(11) - 5.0
    assert len(w) == 11 and abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1], rtol=0, atol=0)
    assert np.argmax(w) == 5 and np.all(np.diff(w[:6]) > 0)
    var = float((w * x * x).sum())
    assert 2.2 < var < 2.25
