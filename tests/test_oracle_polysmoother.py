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


def _columns(op, m, shape):
    """Dense matrix of a linear map on arrays of ``shape`` (m entries), column by column."""
    out = np.zeros((op(np.zeros(shape, dtype=np.complex128)).size, m), dtype=np.complex128)
    for j in range(m):
        e = np.zeros(m, dtype=np.complex128)
        e[j] = 1.0
        out[:, j] = op(e.reshape(shape)).ravel()
    return out


def _taylor_poly_matrix(A, k, h, tb, tg, dim):
    """p(A) = c0 I + c1 (A - t0) + c2 (A - t0)^2 + c3 (A - t0)^3 with the level's phi
    (Eq. polynomial, Taylor form about t0; independent of the factored weights)."""
    phi, _ = PS.level_polynomial(k, h, tb, tg, dim)
    t0, t1, t2 = PS.triangle(k, h, tb, tg, dim)
    e, f = PS.basis_ef(t0, t1, t2)
    c = PS.coefficients(e, f, phi)
    m = A.shape[0]
    S = A - t0 * np.eye(m)
    return c[0] * np.eye(m) + S @ (c[1] * np.eye(m) + S @ (c[2] * np.eye(m) + c[3] * S))


@pytest.mark.parametrize("dim,n", [(2, 7), (2, 15), (3, 7)])
def test_polynomial_vcycle_equals_its_error_propagator(dim, n):
    """With fixed weights the polynomial-smoothed V(1,1) cycle is linear, b -> B b, and
    its error propagator obeys the two-grid recursion of Sec. 3.1 with the smoother's
    e <- p(M) e of Sec. 4.1 on both sides:
        I - B_l M_l = p(M_l) (I - P_l B_{l+1} R_l M_l) p(M_l),   B_coarsest = M^{-1}.
    B is read column by column off ``vcycle_poly``; the right-hand side is built from
    dense matrices, p(M) in its Taylor form."""
    k, tb, tg = 0.2 * (n + 1), np.radians(10.0), np.radians(30.0)
    levels = O.build_hierarchy(dim, n, tb, tg, 0.125, k=k)
    weights = PS.hierarchy_weights(levels, k, tb, tg)
    want = None
    for li in range(len(levels) - 1, -1, -1):
        lev = levels[li]
        M = O.helmholtz.dense_matrix(lev)
        m = M.shape[0]
        if li == len(levels) - 1:
            want = np.linalg.inv(M)
            continue
        nc = levels[li + 1].n
        R = _columns(O.restrict_fw, m, (lev.n,) * dim)
        P = _columns(lambda ec: O.prolong(ec, lev.n), nc ** dim, (nc,) * dim)
        pM = _taylor_poly_matrix(M, k, 1.0 / (lev.n + 1), tb, tg, dim)
        E = pM @ (np.eye(m) - P @ want @ R @ M) @ pM
        want = (np.eye(m) - E) @ np.linalg.inv(M)
    shape = (n,) * dim
    got = _columns(lambda b: PS.vcycle_poly(levels, weights, b), n ** dim, shape)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
    # linearity, the property the closed form rests on
    rng = np.random.default_rng(9)
    b1, b2 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(2))
    lhs = PS.vcycle_poly(levels, weights, 2.0 * b1 - 3.0j * b2)
    rhs = 2.0 * PS.vcycle_poly(levels, weights, b1) - 3.0j * PS.vcycle_poly(levels, weights, b2)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(rhs)
