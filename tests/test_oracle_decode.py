"""Pins for the oracle's direct per-point decode.

The strongest pin is exact polynomial reproduction with control points given in closed
form by Marsden's identity, (y - u)^p = sum_i prod_{j=1..p} (y - t_{i+j}) N_{i,p}(u): the
monomial u^k has B-spline coefficients sigma_k(t_{i+1}, ..., t_{i+p}) / binom(p, k)
(sigma_k the elementary symmetric polynomial). No least-squares fit is involved, so a
wrong index, sign or dropped term anywhere in the basis or the decode fails it.
"""

import itertools
import math

import numpy as np
import pytest

import synth
from oracle import bspline, decode


def marsden_coeffs(t, p, k):
    """B-spline coefficients of u^k for every basis function: sigma_k(t_{i+1..i+p}) / binom(p, k)."""
    C = len(t) - p - 1
    out = np.zeros(C)
    for i in range(C):
        knots = t[i + 1:i + p + 1]
        out[i] = sum(np.prod(c) for c in itertools.combinations(knots, k)) / math.comb(p, k)
    return out


def poly_cps(coef, knots, degrees, ncp):
    """Control points reproducing g(u,v,w) = sum c[m,l,k] u^k v^l w^m (k <= p_x, ...)."""
    (tx, ty, tz), (px, py, pz) = knots, degrees
    P = np.zeros((ncp[2], ncp[1], ncp[0]))
    for m in range(pz + 1):
        for l in range(py + 1):
            for k in range(px + 1):
                P += coef[m, l, k] * np.einsum("c,b,a->cba", marsden_coeffs(tz, pz, m),
                                               marsden_coeffs(ty, py, l), marsden_coeffs(tx, px, k))
    return P


def poly_eval(coef, uvw):
    u, v, w = uvw[:, 0], uvw[:, 1], uvw[:, 2]
    out = np.zeros((len(uvw), 4))
    for m, l, k in itertools.product(*(range(s) for s in coef.shape)):
        c = coef[m, l, k]
        out[:, 0] += c * u ** k * v ** l * w ** m
        out[:, 1] += c * (k * u ** max(k - 1, 0) if k else 0 * u) * v ** l * w ** m
        out[:, 2] += c * u ** k * (l * v ** max(l - 1, 0) if l else 0 * v) * w ** m
        out[:, 3] += c * u ** k * v ** l * (m * w ** max(m - 1, 0) if m else 0 * w)
    return out


def _cases():
    g = synth.rng(21)
    out = []
    for degrees in [(1, 1, 1), (2, 2, 2), (3, 3, 3), (2, 1, 3), (3, 2, 1)]:
        for uniform in (True, False):
            ncp = tuple(int(g.integers(p + 1, p + 7)) for p in degrees)
            knots = tuple(synth.clamped_uniform_knots(C, p) if uniform else synth.random_clamped_knots(C, p, g)
                          for C, p in zip(ncp, degrees))
            out.append((degrees, ncp, knots))
    return out


@pytest.mark.parametrize("degrees,ncp,knots", _cases())
def test_polynomial_reproduction_marsden(degrees, ncp, knots):
    g = synth.rng(7)
    coef = g.uniform(-1, 1, size=(degrees[2] + 1, degrees[1] + 1, degrees[0] + 1))
    P = poly_cps(coef, knots, degrees, ncp)
    uvw = np.concatenate([g.uniform(0, 1, (200, 3)), np.array(list(itertools.product([0.0, 1.0], repeat=3)))])
    got = decode.evaluate_points(P, knots, degrees, uvw)
    want = poly_eval(coef, uvw)
    assert np.max(np.abs(got - want)) < 1e-12


def test_linear_precision_greville():
    """P_a = Greville abscissa xi_a reproduces f(u, v, w) = u exactly (f_u = 1, f_v = f_w = 0)."""
    g = synth.rng(8)
    for p in (1, 2, 3):
        C = 9
        t = synth.random_clamped_knots(C, p, g)
        knots = (t, synth.clamped_uniform_knots(5, 2), synth.clamped_uniform_knots(4, 1))
        P = np.broadcast_to(synth.greville(t, p)[None, None, :], (4, 5, C)).copy()
        uvw = g.uniform(0, 1, (100, 3))
        out = decode.evaluate_points(P, knots, (p, 2, 1), uvw)
        assert np.max(np.abs(out[:, 0] - uvw[:, 0])) < 1e-13
        assert np.max(np.abs(out[:, 1] - 1.0)) < 1e-12
        assert np.max(np.abs(out[:, 2:])) < 1e-12


def test_endpoint_interpolation_and_end_derivative():
    g = synth.rng(9)
    for degrees in [(2, 2, 2), (3, 1, 2)]:
        ncp = (8, 6, 7)
        knots = tuple(synth.random_clamped_knots(C, p, g) for C, p in zip(ncp, degrees))
        P = g.uniform(-1, 1, (ncp[2], ncp[1], ncp[0]))
        for corner in itertools.product([0, 1], repeat=3):
            uvw = np.array([corner], dtype=np.float64)
            f = decode.evaluate_points(P, knots, degrees, uvw)[0, 0]
            a, b, c = (corner[0] * (ncp[0] - 1), corner[1] * (ncp[1] - 1), corner[2] * (ncp[2] - 1))
            assert abs(f - P[c, b, a]) < 1e-14
        # f_u(0, 0, 0) = p / (t_{p+1} - t_1) (P_1 - P_0) along the x edge of a clamped vector
        px, tx = degrees[0], knots[0]
        fu = decode.evaluate_points(P, knots, degrees, np.zeros((1, 3)))[0, 1]
        assert abs(fu - px / (tx[px + 1] - tx[1]) * (P[0, 0, 1] - P[0, 0, 0])) < 1e-12


def test_gradient_matches_finite_differences():
    g = synth.rng(10)
    bs = synth.random_block_set(6, 10, degree_choices=(2, 3), nonuniform=True)
    h = 1e-6
    for b in range(len(bs)):
        P, knots, deg = bs.block_cps(b), bs.block_knots(b), bs.degree[b]
        uvw = g.uniform(0.05, 0.95, (40, 3))
        out = decode.evaluate_points(P, knots, deg, uvw)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            fd = (decode.evaluate_points(P, knots, deg, uvw + e)[:, 0]
                  - decode.evaluate_points(P, knots, deg, uvw - e)[:, 0]) / (2 * h)
            assert np.max(np.abs(fd - out[:, 1 + ax])) < 2e-6 * max(1.0, np.max(np.abs(fd)))


def test_nonzero_terms_equal_full_sum():
    bs = synth.random_block_set(5, 12, nonuniform=True)
    g = synth.rng(12)
    for b in range(len(bs)):
        P, knots, deg = bs.block_cps(b), bs.block_knots(b), bs.degree[b]
        uvw = np.concatenate([g.uniform(0, 1, (30, 3)), [[1.0, 1.0, 1.0], [0.0, 1.0, 0.5]]])
        assert np.max(np.abs(decode.evaluate_points(P, knots, deg, uvw)
                             - decode.evaluate_points_dense(P, knots, deg, uvw))) < 1e-13


def _de_casteljau(coeffs, u):
    c = list(coeffs)
    while len(c) > 1:
        c = [(1 - u) * c[i] + u * c[i + 1] for i in range(len(c) - 1)]
    return c[0]


def test_bezier_case_matches_de_casteljau():
    """C = p + 1 on every axis: the decode is a tensor Bezier volume, evaluated by de Casteljau per axis."""
    g = synth.rng(13)
    for degrees in [(2, 2, 2), (3, 1, 2)]:
        ncp = tuple(p + 1 for p in degrees)
        knots = tuple(synth.clamped_uniform_knots(C, p) for C, p in zip(ncp, degrees))
        P = g.uniform(-1, 1, (ncp[2], ncp[1], ncp[0]))
        for u, v, w in g.uniform(0, 1, (20, 3)):
            along_x = [[_de_casteljau(P[c, b, :], u) for b in range(ncp[1])] for c in range(ncp[2])]
            along_y = [_de_casteljau(row, v) for row in along_x]
            want = _de_casteljau(along_y, w)
            got = decode.evaluate_points(P, knots, degrees, np.array([[u, v, w]]))[0, 0]
            assert abs(got - want) < 1e-14


def test_linear_interpolation_special_case():
    """p = 1 and C = n: the clamped uniform knots sit on the samples, so decode reproduces the control points."""
    g = synth.rng(14)
    n = 9
    knots = tuple(synth.clamped_uniform_knots(n, 1) for _ in range(3))
    P = g.uniform(-1, 1, (n, n, n))
    out = decode.decode_block(P, knots, (1, 1, 1), (n, n, n))
    assert np.max(np.abs(out[..., 0] - P)) < 1e-13  # n - 1 = 8: knots and FP32 sample params are exact
    # forward difference slope inside each interval: f_u = (n - 1) (P[a+1] - P[a]) on [u_a, u_{a+1})
    assert np.max(np.abs(out[:, :, :-1, 1] - (n - 1) * (P[:, :, 1:] - P[:, :, :-1]))) < 1e-12


def test_decode_voxels_matches_decode_block_anisotropic():
    """Selected voxels (k, j, i) decode to the same rows as the whole-grid decode indexed there, on an
    anisotropic grid where any swap of the (k, j, i) -> (u, v, w) mapping lands on other samples."""
    g = synth.rng(43)
    degrees, ncp, n = (2, 3, 1), (5, 6, 4), (7, 11, 5)
    knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
    P = g.uniform(-1, 1, (ncp[2], ncp[1], ncp[0]))
    full = decode.decode_block(P, knots, degrees, n)
    kji = np.stack([g.integers(0, n[2], 60), g.integers(0, n[1], 60), g.integers(0, n[0], 60)], axis=1)
    kji = np.concatenate([kji, [[0, 0, 0], [n[2] - 1, n[1] - 1, n[0] - 1], [n[2] - 1, 0, n[0] - 1]]])
    sel = decode.decode_voxels(P, knots, degrees, n, kji)
    assert np.array_equal(sel, full[kji[:, 0], kji[:, 1], kji[:, 2]])


def test_evaluate_points_multi_matches_per_block():
    """Points of several blocks evaluated together equal each block's own evaluation."""
    g = synth.rng(44)
    degrees, ncp = (3, 2, 1), (6, 4, 5)
    knots = tuple(synth.random_clamped_knots(C, p, g, min_gap=0.1) for C, p in zip(ncp, degrees))
    Ps = g.uniform(-1, 1, (4, ncp[2], ncp[1], ncp[0]))
    uvw = np.concatenate([g.uniform(0, 1, (50, 3)), [[0, 0, 0], [1, 1, 1], [1, 0, 1]]])
    which = g.integers(0, 4, len(uvw))
    got = decode.evaluate_points_multi(Ps, which, knots, degrees, uvw)
    for b in range(4):
        sel = which == b
        assert np.array_equal(got[sel], decode.evaluate_points(Ps[b], knots, degrees, uvw[sel]))


def test_grid_params_order_and_corners():
    """Sample parameters of a block: x fastest, then y, then z; endpoints 0 and 1 on every axis; each
    parameter i/(n-1) rounded to FP32 (the reading both sides take)."""
    nsamp = (3, 4, 5)
    G = decode.grid_params(nsamp)
    assert G.shape == (60, 3)
    assert np.array_equal(G[0], [0, 0, 0]) and np.array_equal(G[-1], [1, 1, 1])
    third = float(np.float32(1 / 3))
    assert np.array_equal(G[1], [0.5, 0, 0]) and np.array_equal(G[3], [0, third, 0]) and G[12][2] == 0.25
    k, j, i = 2, 1, 2
    assert np.array_equal(G[(k * 4 + j) * 3 + i], [np.float32(i / 2), np.float32(j / 3), np.float32(k / 4)])


@pytest.mark.parametrize("axes", [(0, 1, 2), (3, 4, 0), (1, 1, 4), (2, 3, 1)])
def test_polynomial_reproduction_with_repeated_knots(axes):
    """Marsden's identity on knot vectors with repeated interior knots (multiplicity up to p): every polynomial
    of degree <= p per axis is reproduced exactly, value and gradient."""
    knots = tuple(synth.repeated_knots(a) for a in axes)
    degrees = tuple(synth.REPEATED_KNOT_AXES[a][1] for a in axes)
    ncp = tuple(synth.REPEATED_KNOT_AXES[a][0] for a in axes)
    g = synth.rng(71)
    coef = g.uniform(-1, 1, size=(degrees[2] + 1, degrees[1] + 1, degrees[0] + 1))
    P = poly_cps(coef, knots, degrees, ncp)
    inner = np.unique(np.concatenate(knots))
    uvw = np.concatenate([g.uniform(0, 1, (200, 3)), np.stack([inner] * 3, axis=1)])
    assert np.max(np.abs(decode.evaluate_points(P, knots, degrees, uvw) - poly_eval(coef, uvw))) < 1e-11
