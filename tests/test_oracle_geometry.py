"""Pins of the shell-crossing distance (Sect. 2.6) against brute force.

The oracle takes the root of |x + s mu| = R in closed form; here the crossing
is found by bisection on the squared radius along the ray, r(s)^2 =
x^2 + 2 x mu s + s^2, whose sign is evaluated exactly in rational arithmetic,
so the reference shares no formula (and no rounding) with the oracle's root.
"""
from fractions import Fraction

import numpy as np

import oracle


def _bisect_crossing(x, mu, R, s_lo, s_hi, outward):
    X, M, R2 = Fraction(x), Fraction(mu), Fraction(R) ** 2

    def f(s):
        S = Fraction(s)
        return X * X + 2 * X * M * S + S * S - R2

    lo, hi = s_lo, s_hi
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        v = f(mid)
        if (v < 0) == outward:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _brute_distance(x, mu, xi, xo):
    # inner boundary first: minimum of r^2 along the ray at s* = -x mu
    if mu < 0:
        s_star = -x * mu
        r2min = Fraction(x) ** 2 - (Fraction(x) * Fraction(mu)) ** 2
        if r2min <= Fraction(xi) ** 2:
            return _bisect_crossing(x, mu, xi, 0.0, s_star, outward=False), -1
    s_hi = 4 * xo
    return _bisect_crossing(x, mu, xo, max(0.0, -x * mu), s_hi, outward=True), 1


def test_distance_shell_matches_bisection():
    rng = np.random.default_rng(5)
    xi, xo = 0.0367, 0.0400
    worst = 0.0
    for _ in range(1500):
        x = rng.uniform(xi, xo)
        mu = rng.uniform(-1, 1)
        d, w = oracle.distance_shell(x, mu, xi, xo)
        db, wb = _brute_distance(x, mu, xi, xo)
        assert w == wb
        worst = max(worst, abs(d - db) / db)
    assert worst < 1e-12, worst


def test_distance_shell_edge_cases():
    xi, xo = 0.05, 0.06
    # radial outward from the inner boundary: thickness
    d, w = oracle.distance_shell(xi, 1.0, xi, xo)
    assert w == 1 and abs(d - (xo - xi)) <= 1e-17
    # radial inward from the outer boundary: thickness
    d, w = oracle.distance_shell(xo, -1.0, xi, xo)
    assert w == -1 and abs(d - (xo - xi)) <= 1e-17
    # on the outer boundary moving inward but missing the inner sphere: chord 2 x |mu|
    mu = -0.2
    d, w = oracle.distance_shell(xo, mu, xi, xo)
    assert w == 1 and abs(d - 2 * xo * abs(mu)) / d < 1e-14
    # grazing: tangent-ish directions near mu -> 0- from the outer edge
    for mu in (-1e-3, -1e-6, -1e-9):
        d, w = oracle.distance_shell(xo, mu, xi, xo)
        assert w == 1 and d >= 0 and abs(d - 2 * xo * abs(mu)) <= 1e-14 * xo
    # a point a rounding step outside the shell moving outward: distance clamps at 0
    d, w = oracle.distance_shell(np.nextafter(xo, 1), 0.5, xi, xo)
    assert w == 1 and d == 0.0
    # tiny steps from the inner boundary moving inward
    x = xi * (1 + 1e-12)
    d, w = oracle.distance_shell(x, -1.0, xi, xo)
    assert w == -1 and abs(d - (x - xi)) / (x - xi) < 1e-3
