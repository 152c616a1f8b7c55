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

Eq. 2 (model size) and Eq. 4 (NCP* selection) are written out as well.
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
