"""The exact inner-product reference of the basis-arithmetic tests, pinned against
rational arithmetic (fractions.Fraction: every binary64 value and product exact)."""
from fractions import Fraction

import numpy as np

from exact_dot import exact_dot, product_terms


def fraction_dot(v, w):
    re = sum(Fraction(a.real) * Fraction(b.real) + Fraction(a.imag) * Fraction(b.imag) for a, b in zip(v, w))
    im = sum(Fraction(a.real) * Fraction(b.imag) - Fraction(a.imag) * Fraction(b.real) for a, b in zip(v, w))
    return re, im


def test_product_terms_are_exact():
    g = np.random.default_rng(5)
    x = g.standard_normal(200) * 2.0 ** g.integers(-40, 40, 200)
    y = g.standard_normal(200) * 2.0 ** g.integers(-40, 40, 200)
    for a, b, t in zip(x, y, np.array(product_terms(x, y)).T):
        assert sum(Fraction(float(u)) for u in t) == Fraction(float(a)) * Fraction(float(b))


def test_exact_dot_is_correctly_rounded():
    g = np.random.default_rng(6)
    n = 300
    mag = 2.0 ** g.integers(-30, 30, n)
    v = (g.standard_normal(n) + 1j * g.standard_normal(n)) * mag
    w = (g.standard_normal(n) + 1j * g.standard_normal(n)) / mag
    w[::7] = 1j * v[::7] * np.where(g.random(len(w[::7])) < 0.5, 1.0, -1.0)  # cancelling terms
    got = exact_dot(v, w)
    re, im = fraction_dot(v, w)
    # correctly rounded: float(Fraction) rounds to nearest
    assert got.real == float(re) and got.imag == float(im)
