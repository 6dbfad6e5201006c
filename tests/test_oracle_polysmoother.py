"""Pins of the third-degree polynomial smoother (Sec. 4) in the oracle, against values
the paper prints.  Its layout for these figures is Sec. 4's: n interior intervals of h
on [0, 1] and m = n/4 ECS intervals outside on each side.  The oracle's grids put the
layers inside a unit box, so that layout is the box of n + 2m intervals with layer
fraction m / (n + 2m), lengths scaled by n / (n + 2m) and k by its inverse (k h is
unchanged; the polynomial conditions are invariant under the common scaling of the
spectrum)."""
import numpy as np
import pytest

import oracle as O
from oracle import polysmoother as PS


def spectrum_2d(n_int, theta_beta, theta_gamma, k):
    """Eigenvalues of the 2D M^CSG of Sec. 4's layout (Kronecker sum of the 1D
    operator's), with the box's k and h."""
    m = n_int // 4
    N = n_int + 2 * m
    a, d, c = O.coefficients_1d(O.spacings(N - 1, m / N, theta_gamma, theta_beta))
    A = np.diag(d) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    lam = np.linalg.eigvals(A)
    kb = k * N / n_int
    return (lam[:, None] + lam[None, :]).ravel() - kb * kb, kb, 1.0 / N


def test_fig_ex1_which_phi_maps_the_spectrum_inside():
    """Fig. ex1 (k = 100, theta_gamma = pi/6, theta_beta = 2 pi/45, h = 1/128): the
    polynomial with phi = 1.2032 degrees maps every eigenvalue of the 2D preconditioner
    inside the unit circle; the zoom's other angles 0.6303, 0.81212 and 1.0122 degrees
    leave some outside."""
    tb, tg, k = 2 * np.pi / 45, np.pi / 6, 100.0
    lam, kb, hb = spectrum_2d(128, tb, tg, k)
    t0, t1, t2 = PS.triangle(kb, hb, tb, tg, 2)
    e, f = PS.basis_ef(t0, t1, t2)

    def worst(phi_deg):
        return np.abs(PS.evaluate(PS.coefficients(e, f, np.radians(phi_deg)), t0, lam)).max()
    assert worst(1.2032) < 1.0
    for phi_deg in (0.6303, 0.81212, 1.0122):
        assert worst(phi_deg) > 1.0


def min_stable_theta_beta(k, h, theta_gamma):
    """Smallest theta_beta (bisection, radians) for which some phi meets both necessary
    conditions, or None if none below 29.9 degrees does."""
    def ok(tb):
        t0, t1, t2 = PS.triangle(k, h, tb, theta_gamma, 2)
        e, f = PS.basis_ef(t0, t1, t2)
        phi = np.radians(np.arange(0.0, 360.0, 0.1))
        return bool(np.any(PS.first_order(e, f, phi, tb) & PS.second_order(e, f, phi, tb)))
    lo, hi = np.radians(0.05), np.radians(29.9)
    if not ok(hi):
        return None
    if ok(lo):
        return lo
    for _ in range(22):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if ok(mid) else (mid, hi)
    return hi


@pytest.mark.parametrize("h", [1 / 32, 1 / 16])
def test_critical_angle_of_fig_critical_parameters(h):
    """Fig. critical_parameters (theta_gamma = pi/6): above about 9.45 degrees every
    wavenumber admits a phi that meets the first- and second-order conditions; the
    height of the problematic region is the same on every level."""
    worst = max(filter(None, (min_stable_theta_beta(k, h, np.pi / 6) for k in np.arange(1.0, 129.0))))
    assert 9.35 <= np.degrees(worst) <= 9.55


def test_fig_hierarchy_every_level_stable():
    """Fig. hierarchy_spectrum_smoother: k = 40, theta_gamma = 30, theta_beta = 10
    degrees, six levels of n = 2^(8-l) interior intervals: with each level's phi the
    polynomial maps that level's spectrum inside the unit circle."""
    tb, tg, k = np.radians(10.0), np.radians(30.0), 40.0
    for level in range(1, 7):
        lam, kb, hb = spectrum_2d(2 ** (8 - level), tb, tg, k)
        t0, t1, t2 = PS.triangle(kb, hb, tb, tg, 2)
        e, f = PS.basis_ef(t0, t1, t2)
        phi = PS.choose_phi(e, f, tb)
        assert phi is not None
        assert np.abs(PS.evaluate(PS.coefficients(e, f, phi), t0, lam)).max() < 1.0


def test_factored_form_matches_the_polynomial():
    """p(t) = prod (1 - w_j t) with the weights from p's roots (Sec. 4.1)."""
    tb, tg = np.radians(10.0), np.radians(30.0)
    phi, w = PS.level_polynomial(20.0, 1 / 64, tb, tg, 2)
    t0, t1, t2 = PS.triangle(20.0, 1 / 64, tb, tg, 2)
    e, f = PS.basis_ef(t0, t1, t2)
    c = PS.coefficients(e, f, phi)
    t = np.array([t0, t1, t2, 0.0, 0.3 * t1 + 0.5 * t2, -50.0 + 3000j])
    prod = np.prod([1 - wj * t for wj in w], axis=0)
    assert np.allclose(prod, PS.evaluate(c, t0, t), rtol=1e-9, atol=1e-9)
    assert abs(PS.evaluate(c, t0, 0.0) - 1) < 1e-12 and abs(PS.evaluate(c, t0, t1)) < 1e-9


def test_polynomial_vcycle_converges_as_a_stationary_iteration():
    """The polynomial-smoothed V-cycle, iterated as x <- x + V(b - M x) on a small 2D
    problem with theta_beta = 10 degrees (every level's polynomial stable), converges
    monotonically to the direct solve (about 0.67 per cycle here)."""
    n, k, tb, tg = 31, 6.0, np.radians(10.0), np.radians(30.0)
    levels = O.build_hierarchy(2, n, tb, tg, 0.125, k=k)
    weights = PS.hierarchy_weights(levels, k, tb, tg)
    rng = np.random.default_rng(4)
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    exact = np.linalg.solve(O.helmholtz.dense_matrix(levels[0]), b.ravel()).reshape(b.shape)
    x = np.zeros_like(b)
    errs = []
    for _ in range(12):
        x = x + PS.vcycle_poly(levels, weights, b - levels[0].apply(x))
        errs.append(np.linalg.norm(x - exact) / np.linalg.norm(exact))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.05 * errs[0]
