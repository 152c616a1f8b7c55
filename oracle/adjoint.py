"""Adjoint of the micro-model decode in FP64 (oracle; test infrastructure only).

For L(P) = 0.5 * sum_s (f_P(u_s) - D_s)^2 the gradient with respect to a control
point is dL/dP[c, b, a] = sum_s r_s N_a(u_s) N_b(v_s) N_c(w_s) with r = f_P - D: the
transpose of the value decode applied to the residual. It drives the least-squares
encode of Algorithm 1's model() when that fit is done by gradient steps.

Each sample scatters its (p+1)^3 nonzero terms into the gradient directly.
"""

import numpy as np

from . import bspline


def adjoint_block(R, knots, degrees, ncp):
    """dP[c, b, a] = sum over samples of R[k, j, i] N_a(u_i) N_b(v_j) N_c(w_k).

    R: (n_z, n_y, n_x) residual on the block's regular grid; ncp: (C_x, C_y, C_z).
    Returns (C_z, C_y, C_x).
    """
    R = np.asarray(R, dtype=np.float64)
    nz, ny, nx = R.shape
    (tx, ty, tz), (px, py, pz) = knots, degrees
    G = np.zeros((ncp[2], ncp[1], ncp[0]))
    ux, uy, uz = bspline.sample_params(nx), bspline.sample_params(ny), bspline.sample_params(nz)
    sx, Nx = bspline.find_span(tx, px, ux), bspline.basis(tx, px, ux)
    sy, Ny = bspline.find_span(ty, py, uy), bspline.basis(ty, py, uy)
    sz, Nz = bspline.find_span(tz, pz, uz), bspline.basis(tz, pz, uz)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    K, J, I, r = K.ravel(), J.ravel(), I.ravel(), R.ravel()
    for dc in range(pz + 1):
        for db in range(py + 1):
            for da in range(px + 1):
                c = sz[K] - pz + dc
                b = sy[J] - py + db
                a = sx[I] - px + da
                w = Nx[I, a] * Ny[J, b] * Nz[K, c] * r
                np.add.at(G, (c, b, a), w)
    return G
