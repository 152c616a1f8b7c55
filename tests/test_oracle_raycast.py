"""Pins for the oracle ray caster (Algorithm 4): closed forms for the camera (centre ray, image
orientation), the ray/box chord and the sample positions, the front-to-back compositing order and its
sums, early termination, opacity correction, transfer-function interpolation and clamping, headlight
shading, trilinear interpolation across bricks, absent bricks and missed rays; the per-sample query
renderer against polynomial fields and the cache renderer; pixel subsets against the full render."""

import numpy as np

import synth
from oracle import raycast


def _volume(B, n, fill):
    """B^3 bricks of n^3 nodes; fill(gx, gy, gz) -> (f, f_u, f_v, f_w) per node (global node coords)."""
    table = np.arange(B ** 3, dtype=np.int32).reshape(B, B, B)
    cache = np.zeros((B ** 3, n, n, n, 4))
    for bz in range(B):
        for by in range(B):
            for bx in range(B):
                k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
                cache[table[bz, by, bx]] = fill(bx * n + i, by * n + j, bz * n + k)
    return cache, table


def _const_tf(rgba, n=16):
    return np.tile(np.asarray(rgba, dtype=np.float32), (n, 1))


def _axis_view(eye, up=(0.0, 1.0, 0.0), **kw):
    return synth.default_view(width=5, height=5, eye=eye, target=(0.0, 0.0, 0.0), up=up, **kw)


def test_constant_field_closed_form():
    B, n = 2, 8
    N = B * n
    cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, 0.5), 0 * x, 0 * x, 0 * x], -1))
    alpha = float(np.float32(0.05))  # the transfer function is stored in FP32
    rgb = np.array([0.2, 0.4, 0.8], dtype=np.float32).astype(np.float64)
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=1.0)
    img = raycast.raycast(cache, table, n, view, _const_tf([*rgb, alpha]))
    _, _, _, K, _ = raycast.ray_setup(view, (N, N, N))
    assert K[2, 2] == N - 1  # box depth 2 at one sample per voxel spacing 2/(N-1)
    A = 1 - (1 - alpha) ** K[2, 2]
    assert abs(img[2, 2, 3] - A) < 1e-12
    assert np.max(np.abs(img[2, 2, :3] - rgb * A)) < 1e-12  # zero gradient: unshaded colour


def test_early_termination_closed_form():
    B, n = 2, 8
    cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, 0.5), 0 * x, 0 * x, 0 * x], -1))
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=0.99)
    img = raycast.raycast(cache, table, n, view, _const_tf([1.0, 1.0, 1.0, 0.5]))
    # A_k = 1 - 2^-k first exceeds 0.99 at k = 7
    assert abs(img[2, 2, 3] - (1 - 2.0 ** -7)) < 1e-15
    assert abs(img[2, 2, 0] - (1 - 2.0 ** -7)) < 1e-15


def test_headlight_shading_closed_form():
    """Linear field along x: a ray along z sees n . d = 0 (ambient only), a ray along x sees |n . d| = 1."""
    B, n = 2, 8
    N = B * n
    slope = 0.01
    cache, table = _volume(B, n, lambda x, y, z: np.stack(
        [0.3 + slope * x, np.full(x.shape, slope * (n - 1)), 0 * x, 0 * x], -1))
    alpha = float(np.float32(0.04))
    rgb = np.array([0.9, 0.5, 0.1], dtype=np.float32).astype(np.float64)
    tf = _const_tf([*rgb, alpha])
    ka, kd, ks = (float(np.float32(x)) for x in (0.3, 0.6, 0.3))
    for eye, up, d in [((0.0, 0.0, 3.0), (0.0, 1.0, 0.0), 0.0), ((3.0, 0.0, 0.0), (0.0, 1.0, 0.0), 1.0)]:
        view = _axis_view(eye, up=up, opacity_max=1.0, ka=ka, kd=kd, ks=ks, shininess=20.0)
        img = raycast.raycast(cache, table, n, view, tf)
        _, _, _, K, _ = raycast.ray_setup(view, (N, N, N))
        A = 1 - (1 - alpha) ** K[2, 2]
        c = rgb * (ka + kd * d) + ks * d ** 20
        assert abs(img[2, 2, 3] - A) < 1e-12
        assert np.max(np.abs(img[2, 2, :3] - c * A)) < 1e-9


def test_absent_bricks_and_misses_are_black():
    B, n = 2, 8
    cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, 0.5), 0 * x, 0 * x, 0 * x], -1))
    tf = _const_tf([1.0, 1.0, 1.0, 0.3])
    tf[0] = 0.0  # value 0 (an absent brick's nodes) is fully transparent
    view = _axis_view((0.0, 0.0, 3.0))
    img = raycast.raycast(cache, np.full_like(table, -1), n, view, tf)
    assert np.all(img == 0)
    away = synth.default_view(width=4, height=4, eye=(0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0))
    assert np.all(raycast.raycast(cache, table, n, away, tf) == 0)


def test_center_pixel_ray_is_view_direction():
    view = synth.default_view(width=7, height=5)
    d, _, _, _, _ = raycast.ray_setup(view, (64, 64, 64))
    fwd = -np.array(view["eye"]) / np.linalg.norm(view["eye"])
    assert np.max(np.abs(d[2, 3] - fwd)) < 1e-6


def test_image_orientation():
    """Eye on +z looking at the origin with up +y: pixel columns grow towards +x and row 0 is the top (+y).
    With the bricks of x > 0 absent the right columns are black and the left ones are not; with the bricks
    of y > 0 absent the top rows are black. (Rays through columns 5..7 of 8 stay at x > 0.27, beyond the
    cells that touch x = 0; likewise rows 0..2 at y > 0.27.)"""
    B, n = 2, 8
    cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, 0.5), 0 * x, 0 * x, 0 * x], -1))
    tf = _const_tf([1.0, 1.0, 1.0, 0.3])
    tf[0] = 0.0  # an absent brick's nodes (value 0) are transparent
    view = synth.default_view(width=8, height=8, eye=(0.0, 0.0, 3.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0))
    right_absent = table.copy()
    right_absent[:, :, 1] = -1  # table[bz, by, bx]
    img = raycast.raycast(cache, right_absent, n, view, tf)
    assert np.all(img[:, 5:] == 0)
    assert np.all(img[:, :3, 3] > 0.1)
    top_absent = table.copy()
    top_absent[:, 1, :] = -1
    img = raycast.raycast(cache, top_absent, n, view, tf)
    assert np.all(img[:3] == 0)
    assert np.all(img[5:, :, 3] > 0.1)


def test_front_to_back_order_and_sample_positions():
    """f = 0.3 + s g_z (node units) seen by the centre ray from +z: sample k sits at node z = N - 3/2 - k (the
    first sample half a step inside the front face), and a transfer function whose red channel is the value
    itself (alpha constant, no shading) gives the front-to-back sum
    C = alpha sum_k r^k f_k = alpha (c0 S0 - s S1), r = 1 - alpha, f_k = c0 - s k, c0 = 0.3 + s (N - 3/2),
    with the closed forms S0 = (1 - r^K)/(1 - r) and S1 = r (1 - K r^(K-1) + (K-1) r^K)/(1 - r)^2."""
    B, n = 2, 8
    N = B * n
    s = 0.03
    cache, table = _volume(B, n, lambda x, y, z: np.stack([0.3 + s * z, 0 * x, 0 * x, s * (n - 1) + 0 * x], -1))
    alpha = float(np.float32(0.05))
    m = 256
    tf = np.stack([np.arange(m) / (m - 1), np.zeros(m), np.zeros(m), np.full(m, alpha)], 1).astype(np.float32)
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=1.0, vmin=0.0, vmax=1.0, ka=1.0, kd=0.0, ks=0.0)
    img = raycast.raycast(cache, table, n, view, tf)
    K = N - 1
    r = 1.0 - alpha
    S0 = (1 - r ** K) / (1 - r)
    S1 = r * (1 - K * r ** (K - 1) + (K - 1) * r ** K) / (1 - r) ** 2
    c0 = 0.3 + s * (N - 1.5)
    assert abs(img[2, 2, 3] - (1 - r ** K)) < 1e-12
    assert abs(img[2, 2, 0] - alpha * (c0 * S0 - s * S1)) < 1e-7
    # the reversed (back-to-front) weighting, or samples on the nodes, would differ by far more
    assert abs(alpha * (c0 * S0 - s * S1) - alpha * ((0.3 + 0.5 * s) * S0 + s * S1)) > 1e-3


def test_opacity_correction_closed_form():
    """Half-voxel steps (step_voxels = 1/2): alpha' = 1 - (1 - alpha)^(1/2) per sample, so a constant field
    gives A = 1 - (1 - alpha)^(K/2) over the K samples of the chord."""
    B, n = 2, 8
    N = B * n
    cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, 0.5), 0 * x, 0 * x, 0 * x], -1))
    alpha = float(np.float32(0.05))
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=1.0, step_voxels=0.5)
    img = raycast.raycast(cache, table, n, view, _const_tf([1.0, 1.0, 1.0, alpha]))
    _, _, _, K, _ = raycast.ray_setup(view, (N, N, N))
    assert K[2, 2] == 2 * (N - 1)
    assert abs(img[2, 2, 3] - (1 - (1 - alpha) ** (K[2, 2] / 2))) < 1e-12


def test_transfer_function_interpolation_and_clamp():
    """A two-entry transfer function over [vmin, vmax] interpolates linearly in the value and clamps
    outside: constant fields at 0.25 and at 2.0 give alpha(0.25) = a0 + 0.25 (a1 - a0) and alpha(1) = a1."""
    B, n = 2, 8
    N = B * n
    a0, a1 = float(np.float32(0.02)), float(np.float32(0.1))
    tf = np.array([[1.0, 0.0, 0.0, a0], [0.0, 0.0, 1.0, a1]], dtype=np.float32)
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=1.0, vmin=0.0, vmax=1.0)
    _, _, _, K, _ = raycast.ray_setup(view, (N, N, N))
    for value, a, rgb in [(0.25, a0 + 0.25 * (a1 - a0), (0.75, 0.0, 0.25)), (2.0, a1, (0.0, 0.0, 1.0))]:
        cache, table = _volume(B, n, lambda x, y, z: np.stack([np.full(x.shape, value), 0 * x, 0 * x, 0 * x], -1))
        img = raycast.raycast(cache, table, n, view, tf)
        A = 1 - (1 - a) ** K[2, 2]
        assert abs(img[2, 2, 3] - A) < 1e-12
        assert np.max(np.abs(img[2, 2, :3] - np.array(rgb) * A)) < 1e-12


def test_trilinear_interpolation_across_bricks_is_exact_for_linear_fields():
    """A field linear in x, f = 0.1 + 0.05 x (node units), seen by the centre ray along z (world x = 0, i.e.
    node x = (N - 1)/2 = 7.5, halfway between the last node of brick 0 and the first of brick 1): every sample
    reads f = 0.1 + 0.05 * 7.5 = 0.475 exactly, and a transfer function linear in the value gives its alpha."""
    B, n = 2, 8
    N = B * n
    cache, table = _volume(B, n, lambda x, y, z: np.stack([0.1 + 0.05 * x, 0 * x, 0 * x, 0 * x], -1))
    a0, a1 = float(np.float32(0.0)), float(np.float32(0.08))
    tf = np.array([[1.0, 1.0, 1.0, a0], [1.0, 1.0, 1.0, a1]], dtype=np.float32)
    view = _axis_view((0.0, 0.0, 3.0), opacity_max=1.0, vmin=0.0, vmax=1.0)
    img = raycast.raycast(cache, table, n, view, tf)
    _, _, _, K, _ = raycast.ray_setup(view, (N, N, N))
    a = a0 + 0.475 * (a1 - a0)
    assert abs(img[2, 2, 3] - (1 - (1 - a) ** K[2, 2])) < 1e-12


def _poly_bricks(B, n, p, C, c0, cx2, cz):
    """Per-brick control points (Marsden's identity) of F(gx, gy, gz) = c0 + cx2 gx^2 + cz gz in global node
    units: on brick (bx, by, bz), g = b n + u (n - 1) per axis, so F is a polynomial of degree <= 2 in u, w."""
    from test_oracle_decode import poly_cps
    t = np.array([0.0] * (p + 1) + [j / (C - p) for j in range(1, C - p)] + [1.0] * (p + 1))
    knots = (t, t, t)
    blocks, table = [], np.full((B, B, B), -1, dtype=np.int32)
    for bz in range(B):
        for by in range(B):
            for bx in range(B):
                coef = np.zeros((p + 1, p + 1, p + 1))
                coef[0, 0, 0] = c0 + cx2 * (bx * n) ** 2 + cz * bz * n
                coef[0, 0, 1] = 2 * cx2 * bx * n * (n - 1)
                coef[0, 0, 2] = cx2 * (n - 1) ** 2
                coef[1, 0, 0] = cz * (n - 1)
                table[bz, by, bx] = len(blocks)
                blocks.append(poly_cps(coef, knots, (p, p, p), (C, C, C)))
    return (lambda k: (blocks[k], knots, (p, p, p))), table


def test_direct_query_reproduces_polynomial_fields_and_blends_gaps():
    """fetch_direct at random points: inside a brick the exact F and its parametric gradient (F' (n - 1));
    in the one-node gap between bricks along x the linear blend of F at the two boundary nodes."""
    B, n, p, C = 3, 6, 2, 5
    c0, cx2, cz = 0.1, 0.003, 0.02
    blocks, table = _poly_bricks(B, n, p, C, c0, cx2, cz)
    g = synth.rng(61).uniform(0, B * n - 1, (400, 3))
    got = raycast.fetch_direct(blocks, table, n, g)
    F = lambda gx, gz: c0 + cx2 * gx ** 2 + cz * gz
    bx = np.minimum(np.floor(g[:, 0] / n), B - 1)
    lx = g[:, 0] - bx * n
    gap = lx > n - 1
    inside = ~gap & ~(g[:, 2] - np.minimum(np.floor(g[:, 2] / n), B - 1) * n > n - 1)
    assert inside.sum() > 100 and (gap & ~(g[:, 2] % n > n - 1)).sum() > 10
    assert np.max(np.abs(got[inside, 0] - F(g[inside, 0], g[inside, 2]))) < 1e-12
    assert np.max(np.abs(got[inside, 1] - 2 * cx2 * g[inside, 0] * (n - 1))) < 1e-11
    assert np.max(np.abs(got[inside, 2])) < 1e-12
    assert np.max(np.abs(got[inside, 3] - cz * (n - 1))) < 1e-12
    xg = gap & ~(g[:, 2] % n > n - 1)  # gap along x only (z inside a brick; y does not matter)
    w = lx[xg] - (n - 1)
    lo, hi = bx[xg] * n + n - 1, (bx[xg] + 1) * n
    want = (1 - w) * F(lo, g[xg, 2]) + w * F(hi, g[xg, 2])
    assert np.max(np.abs(got[xg, 0] - want)) < 1e-12


def test_direct_and_cache_renders_agree_on_linear_fields():
    """A field linear in every axis is reproduced exactly by the models, by the blends in the gaps and by
    trilinear interpolation of its nodes, so the two renderers give the same image."""
    B, n, p, C = 2, 8, 2, 4
    blocks, table = _poly_bricks(B, n, p, C, 0.2, 0.0, 0.03)
    cache = np.zeros((B ** 3, n, n, n, 4))
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for bz in range(B):
        for by in range(B):
            for bx in range(B):
                gz = bz * n + k
                cache[table[bz, by, bx]] = np.stack([0.2 + 0.03 * gz, 0 * gz, 0 * gz, 0 * gz + 0.03 * (n - 1)], -1)
    tf = np.array([[0.9, 0.5, 0.1, 0.0], [0.1, 0.5, 0.9, 0.1]], dtype=np.float32)
    view = synth.default_view(width=12, height=10, opacity_max=1.0)
    a = raycast.raycast(cache, table, n, view, tf)
    b = raycast.raycast_direct(blocks, table, n, view, tf)
    assert np.max(np.abs(a - b)) < 1e-12
    assert a[..., 3].max() > 0.1


def _mixed_volume(seed, B=3, n=6):
    g = synth.rng(seed)
    table = g.permutation(B ** 3).astype(np.int32).reshape(B, B, B)
    table[g.random(table.shape) < 0.2] = -1
    cache = np.zeros((B ** 3, n, n, n, 4))
    cache[..., 0] = g.uniform(0, 1, cache.shape[:-1])
    cache[..., 1:] = g.uniform(-2, 2, cache.shape[:-1] + (3,))
    return cache, table, n


def test_pixel_subset_equals_full_render():
    """Marching only some rays gives exactly those pixels of the full render, with and without early
    termination (the per-ray set-up and the sample sequence of a ray do not depend on the other rays)."""
    cache, table, n = _mixed_volume(51)
    tf = synth.transfer_function(5)
    tf[:, 3] = np.clip(tf[:, 3] * 8, 0, 1)
    for omax in (1.0, 0.9):
        view = synth.default_view(width=23, height=17, opacity_max=omax)
        full = raycast.raycast(cache, table, n, view, tf).reshape(-1, 4)
        pix = synth.rng(52).choice(23 * 17, 60, replace=False)
        sub = raycast.raycast(cache, table, n, view, tf, pixels=pix)
        assert sub.shape == (60, 4)
        assert np.array_equal(sub, full[pix])
        assert (full[:, 3] > 0).sum() > 100


def test_direct_pixel_subset_equals_full_render():
    """The per-sample-query renderer marches a subset of rays exactly as in its full render."""
    g = synth.rng(55)
    B, n, C, p = 2, 6, 4, 2
    knots = tuple(synth.clamped_uniform_knots(C, p) for _ in range(3))
    Ps = g.uniform(0, 1, (B ** 3, C, C, C))
    table = np.arange(B ** 3, dtype=np.int32).reshape(B, B, B)
    table[1, 0, 1] = -1
    tf = synth.transfer_function(8)
    view = synth.default_view(width=15, height=11, opacity_max=0.95)
    models = lambda b: (Ps[b], knots, (p, p, p))  # noqa: E731
    full = raycast.raycast_direct(models, table, n, view, tf).reshape(-1, 4)
    pix = g.choice(15 * 11, 30, replace=False)
    assert np.array_equal(raycast.raycast_direct(models, table, n, view, tf, pixels=pix), full[pix])
    assert (full[:, 3] > 0).sum() > 40


def test_voxel_function_equals_cache_array():
    """A cache given as a function of (slot, iz, iy, ix) renders the same image as the array it reads."""
    cache, table, n = _mixed_volume(53)
    tf = synth.transfer_function(6)
    view = synth.default_view(width=19, height=13, opacity_max=0.95)
    calls = []

    def voxels(slot, iz, iy, ix):
        calls.append(len(slot))
        return cache[slot, iz, iy, ix]

    a = raycast.raycast(cache, table, n, view, tf)
    b = raycast.raycast(voxels, table, n, view, tf)
    assert calls and np.array_equal(a, b)


def test_decoded_nodes_equal_block_decodes():
    """The on-demand node source returns each slot's decode (oracle.decode.decode_block) at the requested
    nodes, rounded to FP32, for two groups of models with different knots, degrees and grids."""
    from oracle import decode
    g = synth.rng(54)
    groups, full = [], {}
    for slots, degrees, ncp, n in (([4, 0, 2], (2, 2, 2), (5, 5, 5), (6, 6, 6)), ([1, 3], (3, 1, 2), (4, 3, 5), (6, 6, 6))):
        knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
        Ps = g.uniform(-1, 1, (len(slots), ncp[2], ncp[1], ncp[0]))
        groups.append((slots, Ps, knots, degrees, n))
        for m, s in enumerate(slots):
            full[s] = decode.decode_block(Ps[m], knots, degrees, n).astype(np.float32)
    voxels = raycast.decoded_nodes(groups, 5)
    slot = g.integers(0, 5, 400)
    iz, iy, ix = g.integers(0, 6, 400), g.integers(0, 6, 400), g.integers(0, 6, 400)
    got = voxels(slot, iz, iy, ix)
    want = np.stack([full[s][z, y, x] for s, z, y, x in zip(slot, iz, iy, ix)]).astype(np.float64)
    assert np.array_equal(got, want)


def test_camera_frame_is_orthonormal_and_oriented():
    """The camera frame: unit forward towards the target, right = forward x up and up = right x forward
    orthonormal (so right x up = -forward), up on the world up's side, and tan of half the field of view."""
    g = synth.rng(21)
    for _ in range(20):
        eye = g.uniform(-3, 3, 3)
        tgt = g.uniform(-0.5, 0.5, 3)
        view = synth.default_view(width=int(g.integers(8, 64)), height=int(g.integers(8, 64)),
                                  eye=tuple(eye), target=tuple(tgt), fov_y_deg=float(g.uniform(10, 90)))
        e, fwd, right, up, tan_w, tan_h = (np.asarray(x, np.float64) for x in raycast.camera_frame(view))
        d = np.float32(tgt).astype(np.float64) - np.float32(eye).astype(np.float64)
        assert np.allclose(fwd, d / np.linalg.norm(d), atol=1e-6)
        for v in (fwd, right, up):
            assert abs(np.linalg.norm(v) - 1.0) < 1e-6
        assert abs(fwd @ right) < 1e-6 and abs(fwd @ up) < 1e-6 and abs(right @ up) < 1e-6
        assert np.allclose(np.cross(right, up), -fwd, atol=1e-6)
        upw = np.asarray(view["up"], np.float64)
        assert up @ upw > 0 and abs(np.linalg.det(np.stack([upw, fwd, up]))) < 1e-6
        assert abs(tan_h - np.tan(np.radians(view["fov_y_deg"]) / 2)) < 1e-6 * max(1.0, tan_h)
        assert abs(tan_w - tan_h * view["width"] / view["height"]) < 1e-6 * max(1.0, tan_w)
