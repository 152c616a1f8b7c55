"""Front-to-back ray casting over a bricked value+gradient cache (oracle; test infrastructure only).

Algorithm 4 of the paper names the per-sample steps of its renderer: sample location,
value query, transfer functions, gradient query, light coefficients, shading, colour
compositing, and termination once the accumulated opacity exceeds O_max. It does not
fix the camera, the sampling, the interpolation or the lighting model; this oracle
uses these readings:

* volume: B_x*B_y*B_z bricks of n^3 nodes, N_a = B_a*n nodes per axis, mapped to
  [-1, 1]^3 per axis (Sec. 5.1.3 rescales every volume to [-1, 1]); node g sits at
  world -1 + 2 g/(N_a - 1);
* a brick-table entry of -1 marks an absent brick: its nodes read as zero;
* camera: pinhole through pixel centres, row 0 at the top;
* ray/box entry and exit by the slab method; samples at t0 + (k + 1/2) dt with
  dt = step * 2/(N_max - 1) (one sample per voxel at step 1);
* node-centred trilinear interpolation of (f, f_u, f_v, f_w), clamped at the edge;
* transfer function: linear interpolation between tf_n RGBA entries over [vmin, vmax],
  opacity corrected as 1 - (1 - a)^step;
* headlight shading: n = grad f / |grad f| in world units, d = |n . ray|,
  c = rgb (ka + kd d) + ks d^shininess; no shading (c = rgb) when |grad f| < 1e-8;
* compositing: C += (1 - A) a c, A += (1 - A) a; stop when A > O_max; black background.

The integers that floating point decides before marching (hit or miss, and the
number of samples) are computed in FP32 with the operation order an FP32 kernel
uses, so that both sides take the same decision; everything after that is FP64.

:func:`raycast_direct` marches the same rays but queries the micro-models themselves at every
sample (value and parametric gradient of the B-spline, as Algorithm 4's value and gradient
queries do), with this reading for non-overlapping bricks: the model of brick b covers nodes
b n .. b n + n - 1 (parameter u = (g - b n)/(n - 1)); in the one-node gap before brick b + 1 the
value is the linear blend, along that axis, of the two models at their boundary (u = 1 of brick b,
u = 0 of brick b + 1), multilinear where the gaps of several axes meet.
"""

import math

import numpy as np

from . import bspline as _bspline
from . import decode as _decode

f32 = np.float32


def camera_frame(view):
    """Host-side camera set-up in FP64, rounded to FP32: (eye, fwd, right, up, tan_w, tan_h)."""
    eye = np.array(view["eye"], dtype=np.float32).astype(np.float64)
    tgt = np.array(view["target"], dtype=np.float32).astype(np.float64)
    upw = np.array(view["up"], dtype=np.float32).astype(np.float64)
    fwd = tgt - eye
    fwd = fwd / math.sqrt(fwd[0] * fwd[0] + fwd[1] * fwd[1] + fwd[2] * fwd[2])
    right = np.array([fwd[1] * upw[2] - fwd[2] * upw[1],
                      fwd[2] * upw[0] - fwd[0] * upw[2],
                      fwd[0] * upw[1] - fwd[1] * upw[0]])
    right = right / math.sqrt(right[0] * right[0] + right[1] * right[1] + right[2] * right[2])
    up = np.array([right[1] * fwd[2] - right[2] * fwd[1],
                   right[2] * fwd[0] - right[0] * fwd[2],
                   right[0] * fwd[1] - right[1] * fwd[0]])
    fov = float(np.float32(view["fov_y_deg"]))
    tan_h = math.tan(fov * math.pi / 360.0)
    tan_w = tan_h * view["width"] / view["height"]
    return (eye.astype(f32), fwd.astype(f32), right.astype(f32), up.astype(f32),
            f32(tan_w), f32(tan_h))


def ray_setup(view, nodes):
    """FP32 per-pixel direction, entry t0, step dt and sample count K (arrays over pixels)."""
    W, H = int(view["width"]), int(view["height"])
    eye, fwd, right, up, tan_w, tan_h = camera_frame(view)
    nmax = max(nodes)
    dt = f32(float(np.float32(view.get("step_voxels", 1.0))) * 2.0 / (nmax - 1))
    py, px = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    sx = ((2 * px + 1).astype(f32) / f32(W) - f32(1.0)) * tan_w
    sy = (f32(1.0) - (2 * py + 1).astype(f32) / f32(H)) * tan_h
    d = [(fwd[a] + sx * right[a]) + sy * up[a] for a in range(3)]
    length = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    d = [d[a] / length for a in range(3)]
    t0 = np.zeros((H, W), dtype=f32)
    t1 = np.full((H, W), np.inf, dtype=f32)
    miss = np.zeros((H, W), dtype=bool)
    for a in range(3):
        nz = d[a] != 0
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (f32(-1.0) - eye[a]) / d[a]
            tb = (f32(1.0) - eye[a]) / d[a]
        near = np.where(nz, np.minimum(ta, tb), f32(-np.inf))
        far = np.where(nz, np.maximum(ta, tb), f32(np.inf))
        outside = (eye[a] < f32(-1.0)) | (eye[a] > f32(1.0))
        miss |= (~nz) & outside
        t0 = np.maximum(t0, near)
        t1 = np.minimum(t1, far)
    hit = (~miss) & (t1 > t0)
    with np.errstate(invalid="ignore"):
        q = (t1 - t0) / dt
        K = np.ceil(q - f32(0.5))
    K = np.where(hit, np.maximum(K, 0), 0).astype(np.int64)
    return np.stack(d, axis=-1), t0, dt, K, eye


def fetch(cache, table, brick_n, g):
    """Trilinear (f, f_u, f_v, f_w) at voxel coordinates g (M, 3) = (gx, gy, gz), FP64.

    cache is an array (slots, n, n, n, 4), or a function voxels(slot, iz, iy, ix) -> (M, 4) that gives the
    nodes of the listed slots on demand (for volumes too large to decode in full)."""
    Bz, By, Bx = table.shape
    N = np.array([Bx * brick_n, By * brick_n, Bz * brick_n])
    g = np.clip(g, 0.0, (N - 1).astype(np.float64))
    i0 = np.minimum(np.floor(g).astype(np.int64), N - 2)
    w = g - i0
    out = np.zeros((len(g), 4))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix, iy, iz = i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz
                slot = table[iz // brick_n, iy // brick_n, ix // brick_n]
                val = np.zeros((len(g), 4))
                ok = slot >= 0
                at = (slot[ok], iz[ok] % brick_n, iy[ok] % brick_n, ix[ok] % brick_n)
                val[ok] = cache(*at) if callable(cache) else cache[at]
                wt = ((w[:, 0] if dx else 1 - w[:, 0]) * (w[:, 1] if dy else 1 - w[:, 1])
                      * (w[:, 2] if dz else 1 - w[:, 2]))
                out += wt[:, None] * val
    return out


def decoded_nodes(groups, nslots):
    """A cache given as a function (see :func:`fetch`): the nodes of decoded micro-models, computed on demand.

    groups: list of (slots, Ps, knots, degrees, nsamp), the models of one group sharing knots, degrees and
    sample grid; Ps (len(slots), C_z, C_y, C_x) holds the control points of the model in each listed slot.
    A node (iz, iy, ix) of a slot is the model's value and parametric gradient at its sample parameters
    (the decode of :mod:`oracle.decode`), rounded to FP32 as a cache stores it."""
    group = np.full(nslots, -1, dtype=np.int64)
    row = np.zeros(nslots, dtype=np.int64)
    params = []
    for gi, (slots, Ps, knots, degrees, nsamp) in enumerate(groups):
        slots = np.asarray(slots, dtype=np.int64)
        group[slots] = gi
        row[slots] = np.arange(len(slots))
        params.append(tuple(_bspline.sample_params(m) for m in nsamp))

    def voxels(slot, iz, iy, ix):
        out = np.zeros((len(slot), 4))
        g = group[slot]
        for gi in np.unique(g):
            if gi < 0:
                raise ValueError("a slot outside every group")
            sel = g == gi
            _, Ps, knots, degrees, _ = groups[gi]
            ux, uy, uz = params[gi]
            uvw = np.stack([ux[ix[sel]], uy[iy[sel]], uz[iz[sel]]], axis=1)
            out[sel] = _decode.evaluate_points_multi(Ps, row[slot[sel]], knots, degrees, uvw)
        return out.astype(np.float32).astype(np.float64)

    return voxels


def transfer(tf, f, vmin, vmax):
    """Linear interpolation of the RGBA transfer function at values f."""
    n = len(tf)
    x = np.clip((f - vmin) / (vmax - vmin), 0.0, 1.0) * (n - 1)
    i0 = np.minimum(np.floor(x).astype(np.int64), n - 2)
    w = (x - i0)[:, None]
    return tf[i0] * (1 - w) + tf[i0 + 1] * w


def raycast(cache, table, brick_n, view, tf, pixels=None):
    """Render an (H, W, 4) premultiplied RGBA image; cache: (slots, n, n, n, 4) as (f, f_u, f_v, f_w), or a
    function of (slot, iz, iy, ix) as in :func:`fetch`. With pixels (flat indices y * W + x), only those rays
    are marched and their (M, 4) colours returned, in the order given."""
    if not callable(cache):
        cache = np.asarray(cache, dtype=np.float64)
    table = np.asarray(table)
    return _march(table.shape, brick_n, view, tf, lambda g: fetch(cache, table, brick_n, g), pixels)


def fetch_direct(blocks, table, brick_n, g):
    """(f, f_u, f_v, f_w) of the micro-models at voxel coordinates g (M, 3), FP64 (reading in the module
    docstring). blocks(b) -> (P (C_z, C_y, C_x), knots (t_x, t_y, t_z), degrees); table[bz, by, bx] is
    the block of a brick or -1 (absent: zero)."""
    Bz, By, Bx = table.shape
    B = np.array([Bx, By, Bz])
    n = brick_n
    g = np.clip(g, 0.0, (B * n - 1).astype(np.float64))
    b = np.minimum(np.floor(g / n).astype(np.int64), B - 1)
    local = g - b * n
    gap = local > n - 1
    u_in = np.minimum(local, n - 1) / (n - 1)
    w = np.where(gap, local - (n - 1), 0.0)
    out = np.zeros((len(g), 4))
    for combo in range(8):
        side = np.array([(combo >> a) & 1 for a in range(3)])
        use = np.all(gap | (side == 0), axis=1)  # side 1 exists only on gap axes
        if not use.any():
            continue
        bb = b + side[None, :]
        uu = np.where(gap, np.where(side[None, :] == 1, 0.0, 1.0), u_in)
        wt = np.prod(np.where(gap, np.where(side[None, :] == 1, w, 1.0 - w), 1.0), axis=1)
        blk = np.full(len(g), -1, dtype=np.int64)
        blk[use] = table[bb[use, 2], bb[use, 1], bb[use, 0]]
        for k in np.unique(blk[use & (blk >= 0)]):
            sel = use & (blk == k)
            P, knots, degrees = blocks(int(k))
            out[sel] += wt[sel, None] * _decode.evaluate_points(P, knots, degrees, uu[sel])
    return out


def raycast_direct(blocks, table, brick_n, view, tf, pixels=None):
    """Render with a per-sample query of the micro-models (see fetch_direct) instead of a decoded cache; with
    pixels, only those rays (as in :func:`raycast`)."""
    table = np.asarray(table)
    return _march(table.shape, brick_n, view, tf, lambda g: fetch_direct(blocks, table, brick_n, g), pixels)


def _march(table_shape, brick_n, view, tf, sample, pixels=None, nodes=None, gscale=None):
    """Front-to-back marching of every pixel's ray (or of the listed pixels' rays only); sample(g) gives
    (f, f_u, f_v, f_w) at voxel coords g. By default the volume is the brick grid (B_a * brick_n nodes per
    axis) and the gradient is parametric per brick; `nodes` and `gscale` (world gradient per sampled
    gradient unit) replace both."""
    tf = np.asarray(tf, dtype=np.float64)
    if nodes is None:
        Bz, By, Bx = table_shape
        nodes = (Bx * brick_n, By * brick_n, Bz * brick_n)
    H, W = int(view["height"]), int(view["width"])
    d, t0, dt, K, eye = ray_setup(view, nodes)
    d = d.reshape(-1, 3).astype(np.float64)
    t0 = t0.ravel().astype(np.float64)
    K = K.ravel()
    if pixels is not None:  # march a subset of the rays: the per-ray set-up above is unchanged
        pixels = np.asarray(pixels, dtype=np.int64).ravel()
        d, t0, K = d[pixels], t0[pixels], K[pixels]
    eye = eye.astype(np.float64)
    dt = float(dt)
    step = float(np.float32(view.get("step_voxels", 1.0)))
    omax = float(np.float32(view["opacity_max"]))
    ka, kd, ks = (float(np.float32(view[k])) for k in ("ka", "kd", "ks"))
    shin = float(np.float32(view["shininess"]))
    vmin, vmax = float(np.float32(view["vmin"])), float(np.float32(view["vmax"]))
    half = np.array([(n - 1) / 2.0 for n in nodes])
    if gscale is None:
        gscale = half / (brick_n - 1)  # d(world)/d(param): parametric gradient -> world gradient

    M = len(K)
    color = np.zeros((M, 3))
    alpha = np.zeros(M)
    active = K > 0
    k = 0
    while active.any():
        idx = np.nonzero(active)[0]
        t = t0[idx] + (k + 0.5) * dt
        pos = eye[None, :] + t[:, None] * d[idx]
        g = (pos + 1.0) * half[None, :]
        s = sample(g)
        rgba = transfer(tf, s[:, 0], vmin, vmax)
        a = rgba[:, 3] if step == 1.0 else 1.0 - (1.0 - rgba[:, 3]) ** step
        grad = s[:, 1:4] * gscale[None, :]
        gl = np.sqrt(np.sum(grad * grad, axis=1))
        lit = gl >= 1e-8
        nd = np.zeros(len(idx))
        nd[lit] = np.abs(np.sum(grad[lit] * d[idx][lit], axis=1)) / gl[lit]
        shade = np.where(lit, ka + kd * nd, 1.0)
        spec = np.where(lit, ks * nd ** shin, 0.0)
        c = rgba[:, :3] * shade[:, None] + spec[:, None]
        wgt = (1.0 - alpha[idx]) * a
        color[idx] += wgt[:, None] * c
        alpha[idx] += wgt
        k += 1
        active[idx] = (k < K[idx]) & (alpha[idx] <= omax)
    out = np.concatenate([color, alpha[:, None]], axis=1)
    return out if pixels is not None else out.reshape(H, W, 4)
