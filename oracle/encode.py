"""Least-squares micro-model fit in FP64 (oracle; test infrastructure only).

The paper's encoder call model(NCP, degree) (Algorithm 1; MFA, Sec. 4.2) fits the
control points of one micro-block to its n_x*n_y*n_z samples and reports the fitting
error; Table 1 states that error as an RMSE. The fit is the least-squares minimiser

    P* = argmin_P  sum_s (f_P(u_s, v_s, w_s) - D_s)^2 .

With samples on a regular grid the design matrix is the Kronecker product
A = N_z (x) N_y (x) N_x of the per-axis collocation matrices N_a[i, c] = N_c(u_i), so

* :func:`fit_dense` solves the definition directly: lstsq on the full (n^3 x C^3) A
  (tiny blocks only);
* :func:`fit_separable` uses the exact identity (A (x) B (x) C)^+ = A^+ (x) B^+ (x) C^+
  for full-column-rank factors: P = D x_1 N_x^+ x_2 N_y^+ x_3 N_z^+, with each
  N_a^+ = (N_a^T N_a)^{-1} N_a^T from a library solve.

Eq. 2 (model size) and Eq. 4 (NCP* selection) are written out as well, and the cross-level
adaptive encoding of Algorithm 1 (Sec. 4.2.3) over levels of detail built by strided
decimation of the field.
"""

import numpy as np

from . import bspline, decode


def collocation(t, p, n):
    """N_a[i, c] = N_{c,p}(u_i) at the block's n regular sample parameters: shape (n, C)."""
    return bspline.basis(t, p, bspline.sample_params(n))


def fit_dense(D, knots, degrees):
    """Plain least squares on the full Kronecker design matrix. D: (n_z, n_y, n_x)."""
    D = np.asarray(D, dtype=np.float64)
    nz, ny, nx = D.shape
    Nx = collocation(knots[0], degrees[0], nx)
    Ny = collocation(knots[1], degrees[1], ny)
    Nz = collocation(knots[2], degrees[2], nz)
    # Row (k, j, i) and column (c, b, a), both x fastest: A = N_z kron N_y kron N_x.
    A = np.kron(Nz, np.kron(Ny, Nx))
    sol, *_ = np.linalg.lstsq(A, D.ravel(), rcond=None)
    return sol.reshape(Nz.shape[1], Ny.shape[1], Nx.shape[1])


def pseudo_inverse(N):
    """(N^T N)^{-1} N^T for a full-column-rank collocation matrix N (n x C): shape (C, n)."""
    return np.linalg.solve(N.T @ N, N.T)


def fit_separable(D, knots, degrees):
    """Least-squares fit through the per-axis pseudo-inverses. D: (n_z, n_y, n_x) -> P: (C_z, C_y, C_x)."""
    D = np.asarray(D, dtype=np.float64)
    nz, ny, nx = D.shape
    Px = pseudo_inverse(collocation(knots[0], degrees[0], nx))
    Py = pseudo_inverse(collocation(knots[1], degrees[1], ny))
    Pz = pseudo_inverse(collocation(knots[2], degrees[2], nz))
    return np.einsum("ck,bj,ai,kji->cba", Pz, Py, Px, D, optimize=True)


def residual(P, D, knots, degrees):
    """decode(P) - D on the block's sample grid (value channel only)."""
    nz, ny, nx = np.shape(D)
    f = decode.decode_block(P, knots, degrees, (nx, ny, nz))[..., 0]
    return f - np.asarray(D, dtype=np.float64)


def rmse(P, D, knots, degrees):
    """Root-mean-square fitting error over the block's samples (Table 1's error metric)."""
    r = residual(P, D, knots, degrees)
    return float(np.sqrt(np.mean(r * r)))


def model_bytes(ncp, degree):
    """Eq. 2: size in bytes of one micro-model file, 1 + ((NCP + degree) * 3 + NCP^3) * 4."""
    return 1 + ((ncp + degree) * 3 + ncp ** 3) * 4


def select_ncp(errors, bound):
    """Eq. 4: the smallest NCP whose error is below the bound.

    errors: mapping NCP -> Error(NCP). Returns None when no NCP meets the bound.
    """
    ok = [c for c, e in errors.items() if e < bound]
    return min(ok) if ok else None


def fit_separable_batch(Dblocks, knots, degrees):
    """:func:`fit_separable` for a stack of blocks that share knots and degrees: (B, n_z, n_y, n_x) -> (B, C_z, C_y, C_x)."""
    D = np.asarray(Dblocks, dtype=np.float64)
    _, nz, ny, nx = D.shape
    Px = pseudo_inverse(collocation(knots[0], degrees[0], nx))
    Py = pseudo_inverse(collocation(knots[1], degrees[1], ny))
    Pz = pseudo_inverse(collocation(knots[2], degrees[2], nz))
    return np.einsum("ck,bj,ai,nkji->ncba", Pz, Py, Px, D, optimize=True)


def lod_blocks(field, n, stride):
    """Micro-blocks of one level of detail: blocks of n*stride samples per axis of a field (Nz, Ny, Nx),
    keeping every stride-th sample. Returns (blocks (B, n, n, n) as [k][j][i], blocks_per_axis (Bx, By, Bz));
    block id = (bz*By + by)*Bx + bx."""
    F = np.asarray(field)
    Nz, Ny, Nx = F.shape
    span = n * stride
    Bx, By, Bz = Nx // span, Ny // span, Nz // span
    out = []
    for bz in range(Bz):
        for by in range(By):
            for bx in range(Bx):
                blk = F[bz * span:(bz + 1) * span:stride, by * span:(by + 1) * span:stride,
                        bx * span:(bx + 1) * span:stride]
                out.append(blk)
    return np.array(out), (Bx, By, Bz)


def cross_level_select(field, n, degree, bound, levels, knots_of=None):
    """Algorithm 1 (cross-level adaptive encoding), coarsest level first.

    The coarsest level searches every micro-block; a finer level searches only the micro-blocks whose
    parent (the coarser block containing them) was complex. A search fits every NCP in [degree + 2, n]
    and takes NCP* by Eq. 4 on the fit's RMSE; the block is simple when NCP* = degree + 2, else complex
    (no NCP below the bound: complex, encoded with NCP = n). Blocks not searched take NCP = degree + 1.
    knots_of(C) gives the knot vector used for C control points (default: clamped uniform).
    Returns a list of dicts (level, ncp, searched, complex, errors {block: {C: RMSE}})."""
    if knots_of is None:
        def knots_of(C):
            inner = [j / (C - degree) for j in range(1, C - degree)]
            return np.array([0.0] * (degree + 1) + inner + [1.0] * (degree + 1))
    cands = list(range(degree + 2, n + 1))
    result, parent_complex, parent_B = [], None, None
    for lvl in range(levels - 1, -1, -1):
        blocks, B = lod_blocks(field, n, 2 ** lvl)
        nb = len(blocks)
        ncp = np.full(nb, degree + 1, dtype=np.int64)
        searched = np.zeros(nb, dtype=bool)
        cplx = np.zeros(nb, dtype=bool)
        errors = {}
        for b in range(nb):
            bx, by, bz = b % B[0], (b // B[0]) % B[1], b // (B[0] * B[1])
            if parent_complex is not None:
                parent = ((bz // 2) * parent_B[1] + by // 2) * parent_B[0] + bx // 2
                if not parent_complex[parent]:
                    continue
            searched[b] = True
            D = blocks[b].astype(np.float64)
            errs = {}
            for C in cands:
                kn = (knots_of(C),) * 3
                P = fit_separable(D, kn, (degree,) * 3)
                errs[C] = rmse(P, D, kn, (degree,) * 3)
            errors[b] = errs
            star = select_ncp(errs, bound)
            ncp[b] = n if star is None else star
            cplx[b] = star != degree + 2
        result.append({"level": lvl, "ncp": ncp, "searched": searched, "complex": cplx, "errors": errors,
                       "blocks_per_axis": B})
        parent_complex, parent_B = cplx, B
    return result
