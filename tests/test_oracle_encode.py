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
