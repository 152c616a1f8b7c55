"""Multi-resolution micro-blocks and their rendering by level of detail (oracle; test infrastructure only).

Sec. 4.2 partitions the volume into blocks for every level of detail (LOD), with neighbouring blocks
sharing one sample on their common boundary (for C0 continuity), and downsamples each block to the
micro-block resolution of its level. Sec. 5.1.3 renders with four LODs chosen per micro-block by the
distance from the point of view to the block's centroid, over the distance ranges [0, 0.8], [0.8, 1.6],
[1.6, 2.4] and [2.4, inf) in a volume rescaled to [-1, 1]^3; the nearest range takes the finest level.
Sec. 5.2 compares rendered images by MSE, PSNR and SSIM.

Readings used here (the paper gives the rules, not the bookkeeping):

* levels l = 0 (finest) .. L-1; level l has B_l = B_0 / 2^l blocks per axis, each covering (n-1) 2^l
  intervals of the finest grid and sampled every 2^l-th node, so a micro-block always has n^3 samples
  and the field has N = B_0 (n-1) + 1 nodes per axis;
* global block ids list level 0 first, each level z-major: id = off_l + (bz B_l + by) B_l + bx;
* selection is top down: a block of level l >= 1 is rendered when its centroid lies at distance >=
  ranges[l-1] from the eye, otherwise its eight children of level l-1 are examined; level 0 is taken
  when no coarser block was. The distance test is an integer decision taken in FP32, one rounded
  operation at a time: c = (2 g0 + E) / (N - 1) - 1 per axis (g0 the block's first node, E its
  extent in nodes), d^2 = ((c_x - e_x)^2 + (c_y - e_y)^2) + (c_z - e_z)^2 against r^2;
* a sample at finest-node coordinates g belongs to the finest block min(floor(g / (n-1)), B_0 - 1)
  per axis, and is the selected model there at u = (g - g0) / E (clamped to [0, 1]); its gradient in
  node units is the parametric gradient over E.
"""

import numpy as np

from . import decode as _decode
from . import raycast as _raycast

f32 = np.float32
DEFAULT_RANGES = (0.8, 1.6, 2.4)


def shared_blocks(field, n, stride):
    """Micro-blocks of one level with shared boundary samples: the field (N_z, N_y, N_x) with N_a - 1 a
    multiple of (n-1) stride is cut into blocks of (n-1) stride intervals whose neighbours share their
    boundary samples; each keeps every stride-th sample, n^3 in all. Returns (blocks (B, n, n, n) as
    [k][j][i], blocks per axis (B_x, B_y, B_z)); block id = (bz B_y + by) B_x + bx."""
    F = np.asarray(field)
    span = (n - 1) * stride
    B = []
    for N in F.shape[::-1]:
        if (N - 1) % span:
            raise ValueError("field size is not a whole number of shared-boundary blocks")
        B.append((N - 1) // span)
    Bx, By, Bz = B
    out = []
    for bz in range(Bz):
        for by in range(By):
            for bx in range(Bx):
                out.append(F[bz * span: bz * span + span + 1: stride, by * span: by * span + span + 1: stride,
                             bx * span: bx * span + span + 1: stride])
    return np.array(out), (Bx, By, Bz)


def level_offsets(B0, levels):
    """First global id of every level (level 0 first) and the total number of blocks."""
    off, acc = [], 0
    for lvl in range(levels):
        Bl = B0 >> lvl
        off.append(acc)
        acc += Bl ** 3
    return off, acc


def block_geometry(bid, B0, n, levels):
    """(level, first node g0 per axis (x, y, z), extent E in finest nodes) of global block id bid."""
    off, total = level_offsets(B0, levels)
    if not 0 <= bid < total:
        raise ValueError("block id outside every level")
    lvl = max(l for l in range(levels) if off[l] <= bid)
    Bl = B0 >> lvl
    local = bid - off[lvl]
    bx, by, bz = local % Bl, (local // Bl) % Bl, local // (Bl * Bl)
    E = (n - 1) << lvl
    return lvl, (bx * E, by * E, bz * E), E


def _far_enough(g0, E, N, eye, r):
    """The FP32 distance test of the module docstring: centroid at distance >= r from the eye."""
    d2 = f32(0.0)
    for a in range(3):
        c = f32(2 * g0[a] + E) / f32(N - 1) - f32(1.0)
        d = c - f32(eye[a])
        d2 = d2 + d * d if a else d * d
    return bool(d2 >= f32(r) * f32(r))


def select_lod(eye, B0, n, levels, ranges=DEFAULT_RANGES):
    """Top-down LOD selection for a point of view: int64 table (B0, B0, B0) [z][y][x] of the global id of the
    block rendered over each finest block (each selected block of level l covers 2^l finest blocks per axis)."""
    if len(ranges) != levels - 1 or B0 % (1 << (levels - 1)):
        raise ValueError("one range per coarse level, and B0 divisible by 2^(levels-1)")
    off, _ = level_offsets(B0, levels)
    N = B0 * (n - 1) + 1
    table = np.full((B0, B0, B0), -1, dtype=np.int64)

    def visit(lvl, bx, by, bz):
        E = (n - 1) << lvl
        if lvl == 0 or _far_enough((bx * E, by * E, bz * E), E, N, eye, ranges[lvl - 1]):
            Bl = B0 >> lvl
            s = 1 << lvl
            table[bz * s:(bz + 1) * s, by * s:(by + 1) * s, bx * s:(bx + 1) * s] = off[lvl] + (bz * Bl + by) * Bl + bx
            return
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    visit(lvl - 1, 2 * bx + cx, 2 * by + cy, 2 * bz + cz)

    top = B0 >> (levels - 1)
    for bz in range(top):
        for by in range(top):
            for bx in range(top):
                visit(levels - 1, bx, by, bz)
    return table


def fetch_lod(models, table, n, levels, g):
    """(f, df/dg_x, df/dg_y, df/dg_z) at finest-node coordinates g (M, 3), FP64, from the selected models;
    models(bid) -> (P (C_z, C_y, C_x), knots (t_x, t_y, t_z), degrees)."""
    B0 = table.shape[0]
    N = B0 * (n - 1) + 1
    g = np.clip(np.asarray(g, dtype=np.float64), 0.0, N - 1.0)
    fb = np.minimum(np.floor(g / (n - 1)).astype(np.int64), B0 - 1)
    ids = table[fb[:, 2], fb[:, 1], fb[:, 0]]
    out = np.zeros((len(g), 4))
    for bid in np.unique(ids):
        sel = ids == bid
        _, g0, E = block_geometry(int(bid), B0, n, levels)
        u = np.clip((g[sel] - np.array(g0, dtype=np.float64)) / E, 0.0, 1.0)
        P, knots, degrees = models(int(bid))
        v = _decode.evaluate_points(P, knots, degrees, u)
        v[:, 1:] /= E
        out[sel] = v
    return out


def raycast_lod(models, table, n, levels, view, tf, pixels=None):
    """Algorithm 4 with per-sample queries of the models a LOD selection picked (see fetch_lod): the volume
    of N = B0 (n-1) + 1 nodes per axis on [-1, 1]^3, one sample per finest node spacing."""
    table = np.asarray(table)
    B0 = table.shape[0]
    N = B0 * (n - 1) + 1
    half = (N - 1) / 2.0
    return _raycast._march(None, None, view, tf, lambda g: fetch_lod(models, table, n, levels, g), pixels,
                           nodes=(N, N, N), gscale=np.array([half, half, half]))


def mse(a, b):
    """Mean squared error between two images (every channel of every pixel)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    return float(np.mean(d * d))


def psnr(a, b, peak=1.0):
    """Peak signal-to-noise ratio in dB, 10 log10(peak^2 / MSE); infinite for equal images."""
    m = mse(a, b)
    return float("inf") if m == 0.0 else float(10.0 * np.log10(peak * peak / m))


def gaussian_window(size=11, sigma=1.5):
    """Normalised 1-D Gaussian weights of the structural-similarity window."""
    x = np.arange(size) - (size - 1) / 2.0
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _filter_valid(img, w):
    """Separable weighted sums of every size x size window of a 2-D image (valid windows only)."""
    k = len(w)
    H, W = img.shape
    rows = np.zeros((H - k + 1, W))
    for i in range(k):
        rows += w[i] * img[i:H - k + 1 + i, :]
    out = np.zeros((H - k + 1, W - k + 1))
    for j in range(k):
        out += w[j] * rows[:, j:W - k + 1 + j]
    return out


def ssim(a, b, peak=1.0, size=11, sigma=1.5, k1=0.01, k2=0.03):
    """Structural similarity (the third image metric of Sec. 5.2) in its usual form: per channel, the local
    means, variances and covariance under an 11 x 11 Gaussian window (sigma 1.5) over every valid window,
    SSIM = (2 mu_a mu_b + c1)(2 s_ab + c2) / ((mu_a^2 + mu_b^2 + c1)(s_a^2 + s_b^2 + c2)) with
    c1 = (k1 peak)^2, c2 = (k2 peak)^2, averaged over the windows and then over the channels.
    a, b: (H, W) or (H, W, channels)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 2:
        a, b = a[..., None], b[..., None]
    w = gaussian_window(size, sigma)
    c1, c2 = (k1 * peak) ** 2, (k2 * peak) ** 2
    vals = []
    for ch in range(a.shape[2]):
        x, y = a[..., ch], b[..., ch]
        mx, my = _filter_valid(x, w), _filter_valid(y, w)
        sxx = _filter_valid(x * x, w) - mx * mx
        syy = _filter_valid(y * y, w) - my * my
        sxy = _filter_valid(x * y, w) - mx * my
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(m.mean())
    return float(np.mean(vals))
