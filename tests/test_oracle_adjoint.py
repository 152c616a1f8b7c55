"""Pins for the oracle's adjoint (the transposed decode)."""

import numpy as np

import synth
from oracle import adjoint, decode


def test_dot_product_identity():
    """<decode(P), R> = <P, adjoint(R)> with the independent per-point decode."""
    bs = synth.random_block_set(8, 41, nonuniform=True)
    g = synth.rng(41)
    for b in range(len(bs)):
        P, knots, deg, nsamp = bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b]
        R = g.uniform(-1, 1, (nsamp[2], nsamp[1], nsamp[0]))
        lhs = np.sum(decode.decode_block(P, knots, deg, nsamp)[..., 0] * R)
        rhs = np.sum(P * adjoint.adjoint_block(R, knots, deg, bs.ncp[b]))
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_gradient_of_squared_residual_matches_finite_differences():
    g = synth.rng(42)
    degrees, ncp, nsamp = (2, 2, 2), (4, 4, 4), (8, 8, 8)
    knots = tuple(synth.clamped_uniform_knots(C, p) for C, p in zip(ncp, degrees))
    P = g.uniform(-1, 1, (4, 4, 4))
    D = g.uniform(-1, 1, (8, 8, 8))

    def loss(Q):
        r = decode.decode_block(Q, knots, degrees, nsamp)[..., 0] - D
        return 0.5 * np.sum(r * r)

    r = decode.decode_block(P, knots, degrees, nsamp)[..., 0] - D
    G = adjoint.adjoint_block(r, knots, degrees, ncp)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (3, 3, 3), (2, 0, 1)]:
        E = np.zeros_like(P)
        E[idx] = h
        fd = (loss(P + E) - loss(P - E)) / (2 * h)
        assert abs(fd - G[idx]) < 1e-6 * max(1.0, abs(fd))


def test_dot_product_identity_with_repeated_knots():
    """<decode(P), R> = <P, adjoint(R)> on blocks whose knot vectors repeat interior knots."""
    bs = synth.repeated_knot_set(4, 45, nsamp_choices=(9, 13))
    g = synth.rng(45)
    for b in range(len(bs)):
        P, knots, deg, nsamp = bs.block_cps(b), bs.block_knots(b), bs.degree[b], bs.nsamp[b]
        R = g.uniform(-1, 1, (nsamp[2], nsamp[1], nsamp[0]))
        lhs = np.sum(decode.decode_block(P, knots, deg, nsamp)[..., 0] * R)
        rhs = np.sum(P * adjoint.adjoint_block(R, knots, deg, bs.ncp[b]))
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
