"""Pins for the oracle's B-spline basis (textbook properties and closed forms)."""

import math
import os

import numpy as np
import pytest

import synth
from oracle import bspline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _knot_cases():
    g = synth.rng(11)
    cases = []
    for p in (1, 2, 3):
        for C in (p + 1, p + 2, 7, 12):
            cases.append((synth.clamped_uniform_knots(C, p), p))
            cases.append((synth.random_clamped_knots(C, p, g), p))
    return cases


@pytest.mark.parametrize("t,p", _knot_cases())
def test_partition_of_unity_and_support(t, p):
    u = np.concatenate([[0.0, 1.0], np.linspace(0, 1, 97), synth.rng(3).uniform(0, 1, 50), t[p:-p]])
    N = bspline.basis(t, p, u)
    dN = bspline.basis_deriv(t, p, u)
    assert np.max(np.abs(N.sum(axis=1) - 1.0)) < 1e-14
    assert np.max(np.abs(dN.sum(axis=1))) < 1e-11
    assert N.min() >= -1e-15
    s = bspline.find_span(t, p, u)
    C = len(t) - p - 1
    for m in range(len(u)):
        nz = np.nonzero(np.abs(N[m]) > 0)[0]
        assert nz.min() >= s[m] - p and nz.max() <= s[m]
        # span definition: t_s <= u < t_{s+1}, or the last non-empty span at u = 1
        if u[m] < t[C]:
            assert t[s[m]] <= u[m] < t[s[m] + 1]
        else:
            assert s[m] == C - 1


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bernstein_reduction(p):
    """With C = p + 1 the clamped basis is the Bernstein basis B_{i,p}(u) = binom(p, i) u^i (1-u)^(p-i)."""
    t = synth.clamped_uniform_knots(p + 1, p)
    u = np.linspace(0, 1, 41)
    N = bspline.basis(t, p, u)
    dN = bspline.basis_deriv(t, p, u)
    for i in range(p + 1):
        B = math.comb(p, i) * u ** i * (1 - u) ** (p - i)
        assert np.max(np.abs(N[:, i] - B)) < 1e-14
        # d/du B_{i,p} = p (B_{i-1,p-1} - B_{i,p-1})
        lo = math.comb(p - 1, i - 1) * u ** (i - 1) * (1 - u) ** (p - i) if i >= 1 else 0 * u
        hi = math.comb(p - 1, i) * u ** i * (1 - u) ** (p - 1 - i) if i <= p - 1 else 0 * u
        assert np.max(np.abs(dN[:, i] - p * (lo - hi))) < 1e-12


def test_uniform_closed_forms():
    """Interior basis functions of a uniform clamped vector equal the textbook uniform B-spline pieces."""
    rows = np.loadtxt(os.path.join(GOLDEN, "uniform_bspline_closed_form.txt"))
    for p, x, val in rows:
        p = int(p)
        C = 12
        t = synth.clamped_uniform_knots(C, p)
        h = 1.0 / (C - p)
        i = p + 2  # support [t_i, t_{i+p+1}] lies in the uniform interior
        u = t[i] + x * h
        assert abs(bspline.basis(t, p, [u])[0, i] - val) < 1e-13


@pytest.mark.parametrize("t,p", _knot_cases())
def test_derivative_matches_finite_differences(t, p):
    g = synth.rng(5)
    u = g.uniform(0.01, 0.99, 60)
    # keep FD stencils off knots, where N' is discontinuous for p = 1
    keep = np.min(np.abs(u[:, None] - t[None, :]), axis=1) > 2e-4
    u = u[keep]
    h = 1e-6
    fd = (bspline.basis(t, p, u + h) - bspline.basis(t, p, u - h)) / (2 * h)
    assert np.max(np.abs(fd - bspline.basis_deriv(t, p, u))) < 1e-6 * max(1.0, np.max(np.abs(fd)))


def test_sample_params_are_fp32_quotients():
    for n in (2, 5, 32, 64):
        u = bspline.sample_params(n)
        assert u[0] == 0.0 and u[-1] == 1.0
        assert np.all(u == (np.arange(n, dtype=np.float32) / np.float32(n - 1)).astype(np.float64))


@pytest.mark.parametrize("t,p", _knot_cases())
def test_degree0_indicators_cover_each_parameter_once(t, p):
    """Degree 0: every parameter in [t_0, t_end] lies in exactly one half-open knot interval; empty
    intervals (repeated knots) hold none, and the right end belongs to the last non-empty interval."""
    u = np.concatenate([[0.0, 1.0], t, synth.rng(5).uniform(0, 1, 200)])
    N0 = bspline.degree0(t, u)
    assert N0.shape == (len(u), len(t) - 1)
    assert np.all((N0 == 0) | (N0 == 1)) and np.all(N0.sum(axis=1) == 1)
    empty = np.diff(t) == 0
    assert np.all(N0[:, empty] == 0)
    for r, x in enumerate(u):
        i = int(np.argmax(N0[r]))
        assert t[i] <= x and (x < t[i + 1] or (x == t[-1] and t[i] < t[i + 1] == t[-1]))


def _clamped_with_repeats(data):
    """A clamped knot vector for a random degree p and control-point count C whose interior knots sit on a
    coarse grid, each grid point taken up to p times (so the basis stays continuous and knots repeat)."""
    from hypothesis import strategies as st
    p = data.draw(st.integers(1, 3))
    C = data.draw(st.integers(p + 1, 16))
    need = C - p - 1
    lo = max(2, -(-need // p) + 1)  # enough grid points for multiplicities up to p
    grid = data.draw(st.integers(lo, max(lo, need // 2 + 2)))
    counts = [0] * (grid - 1)
    interior = []
    while len(interior) < need:
        i = data.draw(st.integers(0, grid - 2))
        while counts[i] == p:  # the next grid point that is not yet at multiplicity p
            i = (i + 1) % (grid - 1)
        counts[i] += 1
        interior.append((i + 1) / grid)
    return np.array([0.0] * (p + 1) + sorted(interior) + [1.0] * (p + 1)), p


def test_basis_properties_with_repeated_interior_knots():
    """For clamped knot vectors with repeated interior knots: partition of unity, nonnegativity, at most
    p + 1 contiguous nonzero functions starting at the span minus p, derivatives summing to 0, and linear
    precision (the Greville abscissae as control points reproduce u exactly)."""
    from hypothesis import HealthCheck, given, settings
    from hypothesis import strategies as st

    @settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])
    @given(st.data())
    def check(data):
        t, p = _clamped_with_repeats(data)
        C = len(t) - p - 1
        u = np.concatenate([[0.0, 1.0], np.unique(t), synth.rng(len(t)).uniform(0, 1, 40)])
        N, dN = bspline.basis(t, p, u), bspline.basis_deriv(t, p, u)
        s = bspline.find_span(t, p, u)
        assert np.max(np.abs(N.sum(axis=1) - 1.0)) < 1e-13
        assert N.min() >= 0.0
        assert np.max(np.abs(dN.sum(axis=1))) < 1e-9 * max(1.0, np.abs(dN).max())
        for r in range(len(u)):
            nz = np.nonzero(N[r])[0]
            assert len(nz) <= p + 1 and (len(nz) == 0 or (nz[0] >= s[r] - p and nz[-1] <= s[r]))
        greville = np.array([t[i + 1: i + p + 1].sum() / p for i in range(C)])
        assert np.max(np.abs(N @ greville - u)) < 1e-13

    check()
