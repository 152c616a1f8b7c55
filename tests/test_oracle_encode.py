"""Pins for the oracle's least-squares encode, Eq. 2 and Eq. 4."""

import os

import numpy as np
import pytest

import synth
from oracle import adjoint, decode, encode
from test_oracle_decode import poly_cps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_cases():
    g = synth.rng(31)
    out = []
    for degrees, ncp, nsamp in [((1, 1, 1), (3, 4, 2), (5, 6, 4)), ((2, 2, 2), (4, 3, 5), (7, 6, 8)),
                                ((3, 2, 1), (5, 4, 3), (8, 7, 6)), ((2, 3, 2), (3, 4, 4), (4, 8, 5))]:
        knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
        D = g.uniform(-1, 1, (nsamp[2], nsamp[1], nsamp[0]))
        out.append((degrees, ncp, knots, D))
    return out


@pytest.mark.parametrize("degrees,ncp,knots,D", _tiny_cases())
def test_separable_equals_dense_least_squares(degrees, ncp, knots, D):
    Ps = encode.fit_separable(D, knots, degrees)
    Pd = encode.fit_dense(D, knots, degrees)
    assert Ps.shape == (ncp[2], ncp[1], ncp[0])
    assert np.max(np.abs(Ps - Pd)) < 1e-10 * max(1.0, np.max(np.abs(Pd)))


@pytest.mark.parametrize("degrees,ncp,knots,D", _tiny_cases())
def test_residual_orthogonal_to_basis(degrees, ncp, knots, D):
    """Normal equations: N^T (decode(P*) - D) = 0 at the least-squares solution."""
    P = encode.fit_separable(D, knots, degrees)
    r = encode.residual(P, D, knots, degrees)
    G = adjoint.adjoint_block(r, knots, degrees, ncp)
    assert np.max(np.abs(G)) < 1e-11


def test_polynomial_data_is_fitted_exactly():
    g = synth.rng(32)
    degrees, ncp, n = (2, 3, 2), (6, 7, 5), (16, 12, 9)
    knots = tuple(synth.random_clamped_knots(C, p, g) for C, p in zip(ncp, degrees))
    coef = g.uniform(-1, 1, (degrees[2] + 1, degrees[1] + 1, degrees[0] + 1))
    P_true = poly_cps(coef, knots, degrees, ncp)
    D = decode.decode_block(P_true, knots, degrees, n)[..., 0]
    P = encode.fit_separable(D, knots, degrees)
    assert np.max(np.abs(P - P_true)) < 1e-10
    assert encode.rmse(P, D, knots, degrees) < 1e-13


def test_error_decreases_with_nested_refinement_marschner_lobb():
    """Nested uniform knot spaces (C - p = 2, 4, 8, 16) give non-increasing least-squares error (Sec. 4.2:
    a larger NCP fits more accurately), on the Marschner-Lobb signal of Eq. 5 over a sub-box that 24
    samples per axis resolve."""
    n = 24
    s = np.linspace(0.2, 0.6, n)
    Z, Y, X = np.meshgrid(s, s, s, indexing="ij")
    D = synth.marschner_lobb(X, Y, Z)[0]
    p = 2
    errs = []
    for m in (2, 4, 8, 16):
        C = m + p
        knots = tuple(synth.clamped_uniform_knots(C, p) for _ in range(3))
        P = encode.fit_separable(D, knots, (p, p, p))
        errs.append(encode.rmse(P, D, knots, (p, p, p)))
    assert all(b <= a + 1e-15 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.01 * errs[0]


def test_eq2_model_size_golden():
    for ncp, deg, size in np.loadtxt(os.path.join(GOLDEN, "eq2_model_size.txt"), dtype=np.int64):
        assert encode.model_bytes(int(ncp), int(deg)) == size


def test_eq4_selection():
    errors = {24: 1e-6, 20: 3e-6, 16: 2e-5, 12: 9e-5, 8: 4e-4, 6: 1e-3, 4: 5e-3}
    assert encode.select_ncp(errors, 1e-4) == 12
    assert encode.select_ncp(errors, 1e-2) == 4
    assert encode.select_ncp(errors, 1e-7) is None


def test_marschner_lobb_golden_points():
    rows = np.loadtxt(os.path.join(GOLDEN, "marschner_lobb_points.txt"))
    F, Fx, Fy, Fz = synth.marschner_lobb(rows[:, 0], rows[:, 1], rows[:, 2])
    assert np.max(np.abs(F - rows[:, 3])) < 1e-15
    assert np.max(np.abs(Fz - rows[:, 4])) < 1e-15


def test_marschner_lobb_gradient_matches_finite_differences():
    g = synth.rng(33)
    p = g.uniform(-0.9, 0.9, (50, 3))
    _, Fx, Fy, Fz = synth.marschner_lobb(p[:, 0], p[:, 1], p[:, 2])
    h = 1e-6
    for ax, an in enumerate((Fx, Fy, Fz)):
        e = np.zeros(3)
        e[ax] = h
        a = synth.marschner_lobb(*(p + e).T)[0]
        b = synth.marschner_lobb(*(p - e).T)[0]
        assert np.max(np.abs((a - b) / (2 * h) - an)) < 1e-6


def test_lod_blocks_closed_form():
    """Level of detail with stride s: sample (i, j, k) of block (bx, by, bz) is the field at
    ((bx n + i) s, (by n + j) s, (bz n + k) s); with f = x + 10 y + 100 z that is a closed form."""
    N, n, s = 24, 3, 4
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    F = x + 10.0 * y + 100.0 * z
    blocks, B = encode.lod_blocks(F, n, s)
    assert B == (2, 2, 2) and blocks.shape == (8, n, n, n)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for b in range(8):
        bx, by, bz = b % 2, (b // 2) % 2, b // 4
        want = (bx * n + i) * s + 10.0 * (by * n + j) * s + 100.0 * (bz * n + k) * s
        assert np.array_equal(blocks[b], want)


def test_cross_level_constant_half_is_never_refined():
    """Algorithm 1 on a field that is constant for z < N/2 and random for z >= N/2 (n = 4, degree 1,
    NCP in [3, 4]): constant blocks are fitted exactly by any NCP, so they are simple (NCP* = 3) at the
    coarsest level and their descendants are never searched (NCP = degree + 1 = 2); random blocks need
    the interpolating NCP = n = 4 (zero error), so they are complex and every level refines them."""
    N, n, p = 32, 4, 1
    F = np.full((N, N, N), 0.5)
    F[N // 2:] = synth.rng(44).uniform(0, 1, (N // 2, N, N))
    res = encode.cross_level_select(F, n, p, 1e-3, levels=3)
    assert [r["level"] for r in res] == [2, 1, 0]
    for r in res:
        Bx, By, Bz = r["blocks_per_axis"]
        bz = np.arange(Bx * By * Bz) // (Bx * By)
        upper = bz >= Bz // 2
        if r["level"] == 2:
            assert r["searched"].all()
        else:
            assert np.array_equal(r["searched"], upper)
        assert np.array_equal(r["complex"], upper)
        assert np.all(r["ncp"][upper] == n)
        lower_searched = ~upper & r["searched"]
        assert np.all(r["ncp"][lower_searched] == p + 2)
        assert np.all(r["ncp"][~r["searched"]] == p + 1)
        for b, errs in r["errors"].items():
            if not upper[b]:
                assert max(errs.values()) < 1e-12
            else:
                assert errs[n] < 1e-12 and errs[p + 2] > 1e-3


def test_cross_level_searches_exactly_the_children_of_complex_blocks():
    g = synth.rng(45)
    N, n, p = 48, 6, 2
    F = g.uniform(0, 1, (N, N, N))
    F[:, : N // 2] = np.linspace(0, 1, N)[None, None, :]  # linear in x: exactly fitted, simple
    res = encode.cross_level_select(F, n, p, 1e-2, levels=3)
    for coarse, fine in zip(res[:-1], res[1:]):
        Bx, By, Bz = fine["blocks_per_axis"]
        ids = np.arange(Bx * By * Bz)
        bx, by, bz = ids % Bx, (ids // Bx) % By, ids // (Bx * By)
        cB = coarse["blocks_per_axis"]
        parent = ((bz // 2) * cB[1] + by // 2) * cB[0] + bx // 2
        assert np.array_equal(fine["searched"], coarse["complex"][parent])
    assert any(r["complex"].any() for r in res) and any((~r["complex"] & r["searched"]).any() for r in res)


@pytest.mark.parametrize("delta", [0.3, -2.5e-3])
def test_rmse_of_a_known_offset(delta):
    """RMSE (Table 1) of data that differ from the model by +-delta at every sample is exactly |delta|:
    a sum instead of a mean, a mean over n instead of n^3, or a missing square root all fail."""
    g = synth.rng(41)
    degrees, ncp, n = (2, 3, 1), (5, 6, 3), (7, 5, 9)
    knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
    P = g.uniform(-1, 1, (ncp[2], ncp[1], ncp[0]))
    f = decode.decode_block(P, knots, degrees, n)[..., 0]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    s = np.where((i + 2 * j + 3 * k) % 2 == 0, 1.0, -1.0)
    assert abs(s.sum()) > 0  # unbalanced: averaging r before squaring would not give |delta| either
    D = f + delta * s
    assert abs(encode.rmse(P, D, knots, degrees) - abs(delta)) < 1e-14


def test_rmse_golden_trilinear():
    """A residual worked by hand on a 3x2x2 trilinear model (tests/golden/rmse_trilinear_3x2x2.txt)."""
    path = os.path.join(GOLDEN, "rmse_trilinear_3x2x2.txt")
    rows = np.loadtxt(path)
    expected = float([ln for ln in open(path) if ln.startswith("# rmse")][0].split()[2])
    D = np.zeros((2, 2, 3))
    for k, j, i, v in rows:
        D[int(k), int(j), int(i)] = v
    P = np.array([[[1 + 2 * a + 3 * b + 4 * c for a in (0, 1)] for b in (0, 1)] for c in (0, 1)], dtype=float)
    knots = (np.array([0.0, 0.0, 1.0, 1.0]),) * 3
    assert abs(encode.rmse(P, D, knots, (1, 1, 1)) - expected) < 1e-15


def test_fit_separable_batch_matches_per_block_and_dense():
    """The batched fit equals the per-block separable fit on every block, and the dense Kronecker
    least squares (the definition) on tiny blocks."""
    g = synth.rng(42)
    degrees, ncp, n = (2, 1, 3), (4, 3, 5), (6, 5, 8)
    knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
    D = g.uniform(-1, 1, (5, n[2], n[1], n[0]))
    Pb = encode.fit_separable_batch(D, knots, degrees)
    assert Pb.shape == (5, ncp[2], ncp[1], ncp[0])
    for b in range(len(D)):
        Ps = encode.fit_separable(D[b], knots, degrees)
        Pd = encode.fit_dense(D[b], knots, degrees)
        assert np.max(np.abs(Pb[b] - Ps)) < 1e-12
        assert np.max(np.abs(Pb[b] - Pd)) < 1e-10


@pytest.mark.parametrize("C,p,n", [(4, 2, 8), (12, 2, 32), (16, 3, 32), (24, 3, 64), (5, 1, 13)])
def test_collocation_rows_and_pseudo_inverse(C, p, n):
    """The collocation matrix has one row per sample that sums to 1 with at most p + 1 contiguous nonzeros,
    and the pseudo-inverse from the normal equations is a left inverse equal to the SVD-based one."""
    t = synth.clamped_uniform_knots(C, p)
    N = encode.collocation(t, p, n)
    assert N.shape == (n, C)
    assert np.max(np.abs(N.sum(axis=1) - 1.0)) < 1e-14
    for row in N:
        nz = np.nonzero(row)[0]
        assert len(nz) <= p + 1 and np.all(np.diff(nz) == 1)
    A = encode.pseudo_inverse(N)
    assert A.shape == (C, n)
    assert np.max(np.abs(A @ N - np.eye(C))) < 1e-10
    assert np.max(np.abs(A - np.linalg.pinv(N))) < 1e-9 * max(1.0, np.abs(A).max())


@pytest.mark.parametrize("axes,nsamp", [((2, 4, 0), (11, 12, 13)), ((0, 2, 4), (13, 9, 10))])
def test_fit_with_repeated_knots(axes, nsamp):
    """Knot vectors with repeated interior knots: the separable fit equals the dense least squares, its
    residual is orthogonal to the basis, and polynomial data of degree <= p is fitted exactly."""
    knots = tuple(synth.repeated_knots(a) for a in axes)
    degrees = tuple(synth.REPEATED_KNOT_AXES[a][1] for a in axes)
    ncp = tuple(synth.REPEATED_KNOT_AXES[a][0] for a in axes)
    g = synth.rng(73)
    D = g.uniform(-1, 1, (nsamp[2], nsamp[1], nsamp[0]))
    Ps, Pd = encode.fit_separable(D, knots, degrees), encode.fit_dense(D, knots, degrees)
    assert np.max(np.abs(Ps - Pd)) < 1e-10 * max(1.0, np.abs(Pd).max())
    G = adjoint.adjoint_block(encode.residual(Ps, D, knots, degrees), knots, degrees, ncp)
    assert np.max(np.abs(G)) < 1e-11
    coef = g.uniform(-1, 1, (degrees[2] + 1, degrees[1] + 1, degrees[0] + 1))
    P_true = poly_cps(coef, knots, degrees, ncp)
    Dp = decode.decode_block(P_true, knots, degrees, nsamp)[..., 0]
    assert np.max(np.abs(encode.fit_separable(Dp, knots, degrees) - P_true)) < 1e-10
