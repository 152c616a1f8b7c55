"""Direct FP64 evaluation of a trivariate tensor-product B-spline micro-model (oracle).

The model of one micro-block (Sec. 4.2; queried by valueMicroModel and
gradientMicroModel in Algorithm 4) is

    f(u, v, w)  = sum_{a,b,c} N_a(u) N_b(v) N_c(w) P[c, b, a]
    f_u         = sum N'_a(u) N_b(v) N_c(w) P[c, b, a]     (likewise f_v, f_w)

with P stored as an array of shape (C_z, C_y, C_x) (x fastest in memory), knots
t_x, t_y, t_z and degrees p_x, p_y, p_z. Gradients are derivatives with respect to
the block parameters (u, v, w) in [0, 1]^3.

Each point is evaluated on its own: its span per axis, the p+1 nonzero basis values
there, and the (p_x+1)(p_y+1)(p_z+1) products summed term by term. There is no
separable staging; :func:`evaluate_points_dense` sums all C_x*C_y*C_z terms instead and
is used to check the span bookkeeping.
"""

import numpy as np

from . import bspline


def _axis_terms(t, p, u):
    """Per point: first nonzero index s-p, and the p+1 values N, N' starting there."""
    s = bspline.find_span(t, p, u)
    N = bspline.basis(t, p, u)
    dN = bspline.basis_deriv(t, p, u)
    rows = np.arange(len(u))[:, None]
    cols = (s - p)[:, None] + np.arange(p + 1)[None, :]
    return s - p, N[rows, cols], dN[rows, cols]


def evaluate_points(P, knots, degrees, uvw):
    """Value and parametric gradient at arbitrary points.

    P: (C_z, C_y, C_x) control points; knots: (t_x, t_y, t_z); degrees: (p_x, p_y, p_z);
    uvw: (M, 3) parameter coordinates in [0, 1]. Returns (M, 4): f, f_u, f_v, f_w.
    """
    P = np.asarray(P, dtype=np.float64)
    uvw = np.atleast_2d(np.asarray(uvw, dtype=np.float64))
    (tx, ty, tz), (px, py, pz) = knots, degrees
    ox, Nx, dNx = _axis_terms(tx, px, uvw[:, 0])
    oy, Ny, dNy = _axis_terms(ty, py, uvw[:, 1])
    oz, Nz, dNz = _axis_terms(tz, pz, uvw[:, 2])
    out = np.zeros((len(uvw), 4))
    for dc in range(pz + 1):
        for db in range(py + 1):
            for da in range(px + 1):
                cp = P[oz + dc, oy + db, ox + da]
                out[:, 0] += Nx[:, da] * Ny[:, db] * Nz[:, dc] * cp
                out[:, 1] += dNx[:, da] * Ny[:, db] * Nz[:, dc] * cp
                out[:, 2] += Nx[:, da] * dNy[:, db] * Nz[:, dc] * cp
                out[:, 3] += Nx[:, da] * Ny[:, db] * dNz[:, dc] * cp
    return out


def evaluate_points_multi(Ps, which, knots, degrees, uvw):
    """:func:`evaluate_points` for points that belong to several blocks with the same knots and degrees.

    Ps: (B, C_z, C_y, C_x) control points of the blocks; which: (M,) block of each point. Returns (M, 4)."""
    Ps = np.asarray(Ps, dtype=np.float64)
    which = np.asarray(which, dtype=np.int64)
    uvw = np.atleast_2d(np.asarray(uvw, dtype=np.float64))
    (tx, ty, tz), (px, py, pz) = knots, degrees
    ox, Nx, dNx = _axis_terms(tx, px, uvw[:, 0])
    oy, Ny, dNy = _axis_terms(ty, py, uvw[:, 1])
    oz, Nz, dNz = _axis_terms(tz, pz, uvw[:, 2])
    out = np.zeros((len(uvw), 4))
    for dc in range(pz + 1):
        for db in range(py + 1):
            for da in range(px + 1):
                cp = Ps[which, oz + dc, oy + db, ox + da]
                out[:, 0] += Nx[:, da] * Ny[:, db] * Nz[:, dc] * cp
                out[:, 1] += dNx[:, da] * Ny[:, db] * Nz[:, dc] * cp
                out[:, 2] += Nx[:, da] * dNy[:, db] * Nz[:, dc] * cp
                out[:, 3] += Nx[:, da] * Ny[:, db] * dNz[:, dc] * cp
    return out


def evaluate_points_dense(P, knots, degrees, uvw):
    """Same as :func:`evaluate_points` but summing every control point's term (all C^3)."""
    P = np.asarray(P, dtype=np.float64)
    uvw = np.atleast_2d(np.asarray(uvw, dtype=np.float64))
    (tx, ty, tz), (px, py, pz) = knots, degrees
    Nx, dNx = bspline.basis(tx, px, uvw[:, 0]), bspline.basis_deriv(tx, px, uvw[:, 0])
    Ny, dNy = bspline.basis(ty, py, uvw[:, 1]), bspline.basis_deriv(ty, py, uvw[:, 1])
    Nz, dNz = bspline.basis(tz, pz, uvw[:, 2]), bspline.basis_deriv(tz, pz, uvw[:, 2])
    out = np.zeros((len(uvw), 4))
    Cz, Cy, Cx = P.shape
    for c in range(Cz):
        for b in range(Cy):
            for a in range(Cx):
                out[:, 0] += Nx[:, a] * Ny[:, b] * Nz[:, c] * P[c, b, a]
                out[:, 1] += dNx[:, a] * Ny[:, b] * Nz[:, c] * P[c, b, a]
                out[:, 2] += Nx[:, a] * dNy[:, b] * Nz[:, c] * P[c, b, a]
                out[:, 3] += Nx[:, a] * Ny[:, b] * dNz[:, c] * P[c, b, a]
    return out


def grid_params(nsamp):
    """(n_z*n_y*n_x, 3) parameter coordinates (u, v, w) of a block's regular samples, x fastest."""
    nx, ny, nz = nsamp
    u, v, w = bspline.sample_params(nx), bspline.sample_params(ny), bspline.sample_params(nz)
    W, V, U = np.meshgrid(w, v, u, indexing="ij")
    return np.stack([U.ravel(), V.ravel(), W.ravel()], axis=1)


def decode_block(P, knots, degrees, nsamp):
    """Decode one micro-block on its regular grid: returns (n_z, n_y, n_x, 4) = (f, f_u, f_v, f_w)."""
    nx, ny, nz = nsamp
    return evaluate_points(P, knots, degrees, grid_params(nsamp)).reshape(nz, ny, nx, 4)


def decode_voxels(P, knots, degrees, nsamp, kji):
    """Decode selected voxels (rows of (k, j, i) sample indices) of one block: (M, 4)."""
    kji = np.atleast_2d(np.asarray(kji, dtype=np.int64))
    nx, ny, nz = nsamp
    ux, uy, uz = bspline.sample_params(nx), bspline.sample_params(ny), bspline.sample_params(nz)
    uvw = np.stack([ux[kji[:, 2]], uy[kji[:, 1]], uz[kji[:, 0]]], axis=1)
    return evaluate_points(P, knots, degrees, uvw)
