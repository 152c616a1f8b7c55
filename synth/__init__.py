"""Seeded synthetic inputs for the micro-model workloads.

This module only makes inputs: knot vectors, control-point sets, scalar fields, block
sets, transfer functions, views and visible sets. It holds none of the encode, decode,
adjoint or ray-cast arithmetic; the oracle and the CUDA library both receive what it
produces and nothing else.

The paper's datasets (Table 1: Rayleigh-Taylor, Chameleon, Flame, Branch, Rotstrat) and
its recorded 400-POV user trajectories are not available; these seeded fields and orbits
stand in for them with the same block sizes, degrees and NCP ranges:

* ``gm_noise_field``  Gaussian mixture plus band-limited gradient noise (512^3 and 256^3);
* ``flame_field``     turbulent noise with thin tanh fronts (1024^3), standing in for Flame;
* ``marschner_lobb``  the closed-form test signal of Eq. 5 (value and gradient).

Random draws use numpy's PCG64 ``Generator`` seeded from ``BASE_SEED + config``;
lattice gradients of the noise use an integer hash so the fields are identical on the
CPU and the GPU up to floating-point rounding of the smooth parts.
"""

from dataclasses import dataclass, field as dc_field
import math

import numpy as np
import torch

BASE_SEED = 0x240900184


def rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------------------- knots


def clamped_uniform_knots(C, p):
    """Clamped knot vector with uniform interior: p+1 zeros, j/(C-p) for j = 1..C-p-1, p+1 ones."""
    inner = [j / (C - p) for j in range(1, C - p)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1), dtype=np.float64)


def random_clamped_knots(C, p, generator, min_gap=0.02):
    """Clamped knot vector with seeded non-uniform interior knots: the C-p spans get widths
    min_gap + (1 - (C-p) min_gap) * (a Dirichlet(1, ..., 1) draw)."""
    m = C - p  # number of non-empty spans
    gap = min(min_gap, 0.5 / m)
    w = generator.dirichlet(np.ones(m))
    widths = gap + (1.0 - m * gap) * w
    inner = np.cumsum(widths)[:-1]
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def greville(t, p):
    """Greville abscissae xi_i = (t_{i+1} + ... + t_{i+p}) / p: sample sites used to seed control points."""
    t = np.asarray(t, dtype=np.float64)
    C = len(t) - p - 1
    return np.array([t[i + 1:i + p + 1].mean() for i in range(C)])


# ------------------------------------------------------------------------- noise


_GRADS = torch.tensor([
    [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
    [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
    [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1],
    [1, 1, 0], [-1, 1, 0], [0, -1, 1], [0, -1, -1]], dtype=torch.float32)


def _hash3(ix, iy, iz, seed):
    """Integer lattice hash (int64 multiply-xorshift mix); identical on every device."""
    h = ix * 73856093 + iy * 19349663 + iz * 83492791 + ((seed * 2654435761) & 0xFFFFFFFF)
    h = h & 0xFFFFFFFF
    h = (h ^ (h >> 16)) * 0x45D9F3B & 0xFFFFFFFF
    h = (h ^ (h >> 16)) * 0x45D9F3B & 0xFFFFFFFF
    h = h ^ (h >> 16)
    return h & 15


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def gradient_noise(x, y, z, seed):
    """Perlin-style gradient noise (quintic fade, 16-entry edge-gradient table), about [-1, 1]."""
    x0, y0, z0 = torch.floor(x), torch.floor(y), torch.floor(z)
    fx, fy, fz = x - x0, y - y0, z - z0
    ix, iy, iz = x0.long(), y0.long(), z0.long()
    grads = _GRADS.to(x.device, x.dtype)
    u, v, w = _fade(fx), _fade(fy), _fade(fz)
    out = torch.zeros_like(x)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                g = grads[_hash3(ix + dx, iy + dy, iz + dz, seed)]
                dot = g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz)
                wt = (u if dx else 1 - u) * (v if dy else 1 - v) * (w if dz else 1 - w)
                out = out + wt * dot
    return out


def fbm(x, y, z, seed, octaves, base_freq, lacunarity=2.0, gain=0.5, absolute=False):
    """Sum of noise octaves; ``absolute`` sums |noise| (turbulence)."""
    out = torch.zeros_like(x)
    amp, freq = 1.0, base_freq
    for o in range(octaves):
        n = gradient_noise(x * freq, y * freq, z * freq, seed + 101 * o)
        out = out + amp * (n.abs() if absolute else n)
        amp *= gain
        freq *= lacunarity
    return out


def _node_coords(N, z0, z1, device, dtype=torch.float32):
    s = torch.arange(N, device=device, dtype=torch.float64) / (N - 1)
    zs = s[z0:z1]
    Z, Y, X = torch.meshgrid(zs, s, s, indexing="ij")
    return X.to(dtype), Y.to(dtype), Z.to(dtype)


def gaussian_mixture_params(seed, count=8):
    g = rng(seed)
    centers = g.uniform(0.15, 0.85, size=(count, 3))
    sigmas = g.uniform(0.05, 0.2, size=count)
    amps = g.uniform(0.5, 1.0, size=count)
    return centers, sigmas, amps


def gaussian_mixture(X, Y, Z, params):
    centers, sigmas, amps = params
    out = torch.zeros_like(X)
    for (cx, cy, cz), s, a in zip(centers, sigmas, amps):
        r2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
        out = out + a * torch.exp(-r2 / (2.0 * s * s))
    return out


def gm_noise_field(N, seed, device="cpu", noise_amp=0.1, octaves=4, base_freq=4.0, chunk=64):
    """Gaussian mixture + noise_amp * (fbm normalised to [-1, 1]), node-centred on N^3, normalised to [0, 1].

    Returns a float32 tensor of shape (N, N, N) indexed [z, y, x].
    """
    out = torch.empty((N, N, N), dtype=torch.float32, device=device)
    params = gaussian_mixture_params(seed)
    for z0 in range(0, N, chunk):
        X, Y, Z = _node_coords(N, z0, min(N, z0 + chunk), device)
        out[z0:z0 + chunk] = fbm(X, Y, Z, seed, octaves, base_freq)
    out *= noise_amp / out.abs().max()
    for z0 in range(0, N, chunk):
        X, Y, Z = _node_coords(N, z0, min(N, z0 + chunk), device)
        out[z0:z0 + chunk] += gaussian_mixture(X, Y, Z, params)
    lo, hi = out.min(), out.max()
    out -= lo
    out /= hi - lo
    return out


def flame_at(X, Y, Z, N, seed, octaves=6, base_freq=4.0, front_voxels=2.0):
    """Flame stand-in at points (X, Y, Z) in [0, 1]^3 (torch tensors): turbulence T with a tanh front of
    width front_voxels/(N-1) around the level set z = 0.4 + 0.15 T."""
    norm = sum(0.5 ** o for o in range(octaves))
    w = front_voxels / (N - 1)
    T = fbm(X, Y, Z, seed, octaves, base_freq, absolute=True) / norm
    phi = Z - 0.4 - 0.15 * T
    front = 0.5 * (1.0 - torch.tanh(phi / w))
    return 0.8 * front + 0.2 * T


def flame_field(N, seed, device="cpu", octaves=6, base_freq=4.0, front_voxels=2.0, chunk=32):
    """Turbulence with a thin tanh front around the level set z = 0.4 + 0.15 T(x) (stand-in for Flame), on N^3 nodes."""
    out = torch.empty((N, N, N), dtype=torch.float32, device=device)
    for z0 in range(0, N, chunk):
        X, Y, Z = _node_coords(N, z0, min(N, z0 + chunk), device)
        out[z0:z0 + chunk] = flame_at(X, Y, Z, N, seed, octaves, base_freq, front_voxels)
    return out


def greville_cps(field_at, Bdims, n, ncp, degree, device="cpu", max_points=1 << 24):
    """Control points = a field evaluated at the Greville abscissae of each brick (clamped uniform knots).

    field_at(X, Y, Z) takes global coordinates in [0, 1]^3 (node-centred on Bdims*n nodes per axis);
    ncp[b] is the isotropic C of brick b (z-major ids). Returns a list of (C, C, C) float32 arrays."""
    Bx, By, Bz = Bdims
    N = (Bx * n, By * n, Bz * n)
    out = [None] * len(ncp)
    ids = np.arange(len(ncp))
    for C in sorted(set(int(c) for c in ncp)):
        xi = torch.as_tensor(greville(clamped_uniform_knots(C, degree), degree), dtype=torch.float64, device=device)
        sel = ids[np.asarray(ncp) == C]
        per = C ** 3
        step = max(1, max_points // per)
        for s0 in range(0, len(sel), step):
            bb = torch.as_tensor(sel[s0:s0 + step], device=device)
            bz, by, bx = bb // (Bx * By), (bb // Bx) % By, bb % Bx
            Zl, Yl, Xl = torch.meshgrid(xi, xi, xi, indexing="ij")
            gx = (bx[:, None, None, None] * n + Xl[None] * (n - 1)) / (N[0] - 1)
            gy = (by[:, None, None, None] * n + Yl[None] * (n - 1)) / (N[1] - 1)
            gz = (bz[:, None, None, None] * n + Zl[None] * (n - 1)) / (N[2] - 1)
            vals = field_at(gx.float(), gy.float(), gz.float()).cpu().numpy().astype(np.float32)
            for m, b in enumerate(sel[s0:s0 + step]):
                out[b] = vals[m]
    return out


def fov_for_visible(target, bricks_per_axis, frame=0, lo=5.0, hi=120.0, iters=30, **kw):
    """Field of view (degrees) for which about `target` bricks are visible in orbit frame `frame`."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        nvis = len(visible_bricks(orbit_view(frame, fov_y_deg=mid, **kw), bricks_per_axis))
        if nvis < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def marschner_lobb(x, y, z, f_m=6.0, alpha=0.05):
    """Eq. 5: F = (1 - sin(pi z/2) + alpha (1 + rho(sqrt(x^2 + y^2)))) / (2 (1 + alpha)),
    rho(r) = cos(2 pi f_M cos(pi r / 2)). Returns (F, dF/dx, dF/dy, dF/dz), numpy FP64."""
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    r = np.sqrt(x * x + y * y)
    inner = 2.0 * np.pi * f_m * np.cos(np.pi * r / 2.0)
    rho = np.cos(inner)
    F = (1.0 - np.sin(np.pi * z / 2.0) + alpha * (1.0 + rho)) / (2.0 * (1.0 + alpha))
    # d rho / d r = sin(inner) * 2 pi f_M * sin(pi r / 2) * pi / 2
    drho = np.sin(inner) * 2.0 * np.pi * f_m * np.sin(np.pi * r / 2.0) * (np.pi / 2.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        rx = np.where(r > 0, x / r, 0.0)
        ry = np.where(r > 0, y / r, 0.0)
    k = alpha / (2.0 * (1.0 + alpha))
    Fx = k * drho * rx
    Fy = k * drho * ry
    Fz = -np.cos(np.pi * z / 2.0) * (np.pi / 2.0) / (2.0 * (1.0 + alpha))
    return F, Fx, Fy, Fz


def gm_params_field_at(points, seed):
    """Gaussian-mixture value at arbitrary points (M, 3) in [0, 1]^3, numpy FP64 (the single-block control points)."""
    centers, sigmas, amps = gaussian_mixture_params(seed)
    p = np.asarray(points, dtype=np.float64)
    out = np.zeros(len(p))
    for c, s, a in zip(centers, sigmas, amps):
        out += a * np.exp(-np.sum((p - c) ** 2, axis=1) / (2.0 * s * s))
    return out


# ----------------------------------------------------------------------- blocks


def blocks_from_field(field, n):
    """Cut an (N_z, N_y, N_x) field into non-overlapping n^3 bricks: (B, n, n, n), brick id z-major."""
    Nz, Ny, Nx = field.shape
    Bz, By, Bx = Nz // n, Ny // n, Nx // n
    f = field.reshape(Bz, n, By, n, Bx, n).permute(0, 2, 4, 1, 3, 5) if torch.is_tensor(field) \
        else field.reshape(Bz, n, By, n, Bx, n).transpose(0, 2, 4, 1, 3, 5)
    return f.reshape(Bz * By * Bx, n, n, n)


def gradient_energy(blocks):
    """Mean squared central-difference gradient of each block's samples (interior samples): (B,)."""
    b = blocks if torch.is_tensor(blocks) else torch.as_tensor(blocks)
    b = b.float()
    gx = (b[:, 1:-1, 1:-1, 2:] - b[:, 1:-1, 1:-1, :-2]) * 0.5
    gy = (b[:, 1:-1, 2:, 1:-1] - b[:, 1:-1, :-2, 1:-1]) * 0.5
    gz = (b[:, 2:, 1:-1, 1:-1] - b[:, :-2, 1:-1, 1:-1]) * 0.5
    return (gx * gx + gy * gy + gz * gz).mean(dim=(1, 2, 3))


def ncp_by_energy(energy, classes, percentiles):
    """Assign each block the class whose percentile bin holds its energy.

    ``percentiles`` has len(classes) - 1 increasing cut points (in percent); blocks below the
    first cut get classes[0], and so on.
    """
    e = energy.detach().cpu().double().numpy() if torch.is_tensor(energy) else np.asarray(energy)
    cuts = np.percentile(e, percentiles)
    idx = np.searchsorted(cuts, e, side="right")
    return np.asarray(classes)[idx]


FLAME_NCP_CLASSES = (4, 6, 8, 12, 16, 20, 24)
FLAME_NCP_PERCENTILES = (50, 65, 77, 86, 92, 96)


@dataclass
class BlockSet:
    """A batch of micro-blocks in the flat layout the library and the oracle both read.

    knots: float32, every axis' knot vector concatenated; cps: float32, every block's
    C_x*C_y*C_z control points (x fastest) concatenated. Per block: degree, ncp, nsamp
    (x, y, z order), knot_off (x, y, z), cp_off, slot and origin (brick coordinates).
    """
    degree: np.ndarray
    ncp: np.ndarray
    nsamp: np.ndarray
    knot_off: np.ndarray
    cp_off: np.ndarray
    slot: np.ndarray
    origin: np.ndarray
    knots: np.ndarray
    cps: np.ndarray
    meta: dict = dc_field(default_factory=dict)

    def __len__(self):
        return len(self.slot)

    def block_knots(self, b):
        return tuple(self.knots[self.knot_off[b, a]:self.knot_off[b, a] + self.ncp[b, a] + self.degree[b, a] + 1]
                     .astype(np.float64) for a in range(3))

    def block_cps(self, b):
        Cx, Cy, Cz = self.ncp[b]
        o = self.cp_off[b]
        return self.cps[o:o + Cx * Cy * Cz].astype(np.float64).reshape(Cz, Cy, Cx)

    def block_voxels(self, b):
        nx, ny, nz = self.nsamp[b]
        return int(nx * ny * nz)


class KnotPool:
    """Deduplicating store of knot vectors (blocks with equal (C, p) share one uniform vector)."""

    def __init__(self):
        self.vectors, self.index = [], {}
        self.size = 0

    def add(self, t):
        key = tuple(np.asarray(t, dtype=np.float32).tolist())
        if key not in self.index:
            self.index[key] = self.size
            self.vectors.append(np.asarray(key, dtype=np.float32))
            self.size += len(key)
        return self.index[key]

    def array(self):
        return np.concatenate(self.vectors) if self.vectors else np.zeros(0, np.float32)


def make_block_set(ncp, degree, nsamp, cps_list, knots_list=None, slots=None, origins=None, meta=None):
    """Assemble a BlockSet. ncp/degree/nsamp: (B, 3) int; cps_list[b]: (C_z, C_y, C_x) array;
    knots_list[b]: 3 knot vectors (default: clamped uniform)."""
    ncp, degree, nsamp = (np.asarray(a, dtype=np.int32).reshape(-1, 3) for a in (ncp, degree, nsamp))
    B = len(ncp)
    pool = KnotPool()
    knot_off = np.zeros((B, 3), dtype=np.int64)
    for b in range(B):
        for a in range(3):
            t = knots_list[b][a] if knots_list is not None else clamped_uniform_knots(ncp[b, a], degree[b, a])
            knot_off[b, a] = pool.add(t)
    sizes = np.prod(ncp.astype(np.int64), axis=1)
    cp_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    cps = np.concatenate([np.asarray(c, dtype=np.float32).ravel() for c in cps_list]) if B else np.zeros(0, np.float32)
    slot = np.arange(B, dtype=np.int32) if slots is None else np.asarray(slots, dtype=np.int32)
    origin = np.zeros((B, 3), dtype=np.int32) if origins is None else np.asarray(origins, dtype=np.int32)
    return BlockSet(degree, ncp, nsamp, knot_off, cp_off, slot, origin, pool.array(), cps, meta or {})


# Clamped knot vectors whose interior knots repeat (multiplicity up to p), as (C, p, interior knots): spans jump
# over the empty intervals, so a sample's band can move by more than one control point from its neighbour's.
REPEATED_KNOT_AXES = [
    (8, 2, [1 / 4, 1 / 4, 1 / 2, 3 / 4, 3 / 4]),
    (10, 3, [1 / 4, 1 / 4, 1 / 2, 1 / 2, 1 / 2, 3 / 4]),
    (6, 1, [1 / 5, 2 / 5, 3 / 5, 4 / 5]),
    (12, 2, [1 / 8, 1 / 4, 1 / 4, 3 / 8, 1 / 2, 1 / 2, 5 / 8, 3 / 4, 7 / 8]),
    (7, 3, [3 / 8, 3 / 8, 5 / 8]),
]


def repeated_knots(axis):
    """Full clamped knot vector of REPEATED_KNOT_AXES[axis] (float64)."""
    C, p, inner = REPEATED_KNOT_AXES[axis]
    return np.array([0.0] * (p + 1) + list(inner) + [1.0] * (p + 1))


def repeated_knot_set(nblocks, seed, nsamp_choices=(32,)):
    """Blocks whose three axes each take one of REPEATED_KNOT_AXES (seeded), control points U[-1, 1]."""
    g = rng(seed)
    ncp, deg, ns, cps, kn = [], [], [], [], []
    for _ in range(nblocks):
        axes = [int(i) for i in g.integers(0, len(REPEATED_KNOT_AXES), 3)]
        ncp.append([REPEATED_KNOT_AXES[a][0] for a in axes])
        deg.append([REPEATED_KNOT_AXES[a][1] for a in axes])
        ns.append([int(g.choice(nsamp_choices)) for _ in range(3)])
        kn.append([repeated_knots(a) for a in axes])
        cps.append(g.uniform(-1, 1, size=(ncp[-1][2], ncp[-1][1], ncp[-1][0])))
    return make_block_set(ncp, deg, ns, cps, kn)


def random_block_set(B, seed, ncp_choices=(4, 6, 8, 12), degree_choices=(1, 2, 3), nsamp_choices=(5, 8, 13, 32),
                     nonuniform=False, anisotropic=True, min_gap=0.02):
    """Small mixed batch for parity tests: random per-axis (C, p, n) with p+1 <= C <= n, random CPs in [-1, 1]."""
    g = rng(seed)
    ncp, deg, ns, cps, knots = [], [], [], [], []
    for _ in range(B):
        d3, c3, n3, t3 = [], [], [], []
        p_iso = int(g.choice(degree_choices))
        for a in range(3):
            p = int(g.choice(degree_choices)) if anisotropic else p_iso
            n = int(g.choice(nsamp_choices))
            opts = [c for c in ncp_choices if p + 1 <= c <= n] or [p + 1]
            C = int(g.choice(opts))
            d3.append(p), c3.append(C), n3.append(n)
            t3.append(random_clamped_knots(C, p, g, min_gap) if nonuniform else clamped_uniform_knots(C, p))
        ncp.append(c3), deg.append(d3), ns.append(n3), knots.append(t3)
        cps.append(g.uniform(-1.0, 1.0, size=(c3[2], c3[1], c3[0])))
    return make_block_set(ncp, deg, ns, cps, knots)


# ------------------------------------------------------------------- rendering


def transfer_function(seed, n=256, bumps=3):
    """RGBA transfer function: Gaussian opacity bumps over [0, 1] and a smooth colour ramp. (n, 4) float32."""
    g = rng(seed)
    x = np.linspace(0.0, 1.0, n)
    mu = g.uniform(0.2, 0.85, size=bumps)
    sd = g.uniform(0.02, 0.08, size=bumps)
    h = g.uniform(0.02, 0.12, size=bumps)
    a = np.zeros(n)
    for m, s, hh in zip(mu, sd, h):
        a += hh * np.exp(-0.5 * ((x - m) / s) ** 2)
    r = np.clip(1.5 * x, 0, 1)
    gg = 4.0 * x * (1.0 - x)
    b = np.clip(1.0 - 1.5 * x, 0, 1)
    return np.stack([r, gg, b, np.clip(a, 0, 1)], axis=1).astype(np.float32)


def default_view(width=1024, height=1024, **kw):
    v = dict(eye=(2.2, 1.6, 2.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=40.0,
             width=width, height=height, step_voxels=1.0, opacity_max=0.99,
             ka=0.3, kd=0.6, ks=0.3, shininess=20.0, vmin=0.0, vmax=1.0)
    v.update(kw)
    return v


def orbit_view(frame, radius=2.5, elevation_deg=20.0, step_deg=11.25, fov_y_deg=40.0, width=1024, height=1024):
    th = math.radians(step_deg * frame)
    el = math.radians(elevation_deg)
    eye = (radius * math.cos(el) * math.cos(th), radius * math.sin(el), radius * math.cos(el) * math.sin(th))
    return default_view(width, height, eye=eye, fov_y_deg=fov_y_deg)


def visible_bricks(view, bricks_per_axis):
    """Bricks (z-major ids) whose world-space AABB meets the view frustum (conservative plane test)."""
    B = bricks_per_axis
    eye = np.array(view["eye"], dtype=np.float64)
    tgt = np.array(view["target"], dtype=np.float64)
    up = np.array(view["up"], dtype=np.float64)
    f = tgt - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(view["fov_y_deg"]) / 2)
    tw = th * view["width"] / view["height"]
    # Side planes through the eye: inward normals.
    normals = [np.cross(u, f + tw * r), np.cross(f - tw * r, u), np.cross(f + th * u, r), np.cross(r, f - th * u)]
    normals = [n / np.linalg.norm(n) for n in normals]
    edges = np.linspace(-1.0, 1.0, B + 1)
    bz, by, bx = np.meshgrid(np.arange(B), np.arange(B), np.arange(B), indexing="ij")
    lo = np.stack([edges[bx], edges[by], edges[bz]], axis=-1).reshape(-1, 3)
    hi = np.stack([edges[bx + 1], edges[by + 1], edges[bz + 1]], axis=-1).reshape(-1, 3)
    keep = np.ones(len(lo), dtype=bool)
    for n in normals:
        # farthest corner along the normal must be on the inner side
        corner = np.where(n[None, :] >= 0, hi, lo)
        keep &= (corner - eye[None, :]) @ n >= 0
    return np.nonzero(keep)[0].astype(np.int32)
