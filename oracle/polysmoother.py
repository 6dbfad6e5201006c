"""Third-degree polynomial smoother (Sec. 4) for the CSG preconditioner: test
infrastructure only, like the rest of this package.

On a level of real spacing h the spectrum of M^CSG lies in the triangle
t0 t1 t2 of Prop. 3.1 (Sec. 3, Sec. 4.1):

    t0 = -k^2,   t1 = -k^2 + 4d / (h e^{i theta_beta})^2,   t2 = -k^2 + 4d / (h e^{i theta_gamma})^2.

The smoother applies p(M) to the error, p of degree 3 with p(0) = 1 (Eq. polyreq4),
p(t1) = p(t2) = 0 (Eq. polyreq2) and p(t0) = e^{i phi} (Eq. polyreq3).  Written as a
Taylor polynomial about t0 (Eq. polynomial), c0 = e^{i phi} and (c1, c2, c3) solve the
3 x 3 Vandermonde system of Eq. coefficients_system, so c = e - e^{i phi} f
(Eq. coefficients_solution) with e, f the solutions for right-hand sides (1, 0, 0) and
(1, 1, 1).  In factored form p(t) = (1 - w1 t)(1 - w2 t)(1 - w3 t): three Richardson
steps x <- x + w_j (b - M x) with the reciprocals of p's roots (Sec. 4.1).

Readings (the paper's formulas for phi are partly garbled):
* First-order condition (Eq. firstorder_varphi): along the top edge
  t = t0 + rho e^{-2 i theta_beta}, |c0 + c1 rho e^{-2i theta_beta}| < 1 for small rho
  holds iff Re(e^{-i phi} c1 e^{-2 i theta_beta}) < 0, i.e.
  |e1| cos(phi_e - phi - 2 theta_beta) < |f1| cos(phi_f - 2 theta_beta).  The printed
  cos(phi + phi_e - 2 theta_beta) (and the interval derived from it) has the sign of phi
  flipped: with it the critical angle of Fig. critical_parameters comes out near 28
  degrees instead of the printed 9.45.
* Second-order condition (Eq. secondorder_varphi) as printed:
  2 Re((e^{-i phi} e2 - f2) e^{-4 i theta_beta}) + |e1 - e^{i phi} f1|^2 < 0.
* Choice of phi (Sec. 4.5 picks it per level within the allowed range but states no
  rule): the midpoint of the longest arc of phi (on a 0.05 degree grid) meeting both
  conditions; where the first-order condition holds for every phi (the region right of
  the dashed lines in Fig. critical_parameters, unconditional stability) phi = 0; where
  neither applies no stable polynomial exists and ``choose_phi`` returns None.
* Constant k only (the triangle's vertices assume phi = k^2 everywhere).

Parity status: pinned by the paper's printed values and, for the cycle, by its error
propagator in closed form, see ``tests/test_oracle_polysmoother.py``: Fig. ex1 (k = 100, theta_gamma = pi/6,
theta_beta = 2 pi/45, h = 1/128: phi = 1.2032 degrees maps the 2D spectrum inside the
unit circle, 0.6303, 0.81212 and 1.0122 degrees do not), the critical angle of
Fig. critical_parameters (9.45 degrees) and Fig. hierarchy_spectrum_smoother (all six
levels stable at theta_beta = 10 degrees, k = 40).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .helmholtz import Level, coarse_solve, prolong, restrict_fw

PHI_GRID = np.radians(np.arange(0.0, 360.0, 0.05))


def triangle(k: float, h: float, theta_beta: float, theta_gamma: float, dim: int):
    """Vertices t0, t1, t2 of the bounding triangle of the spectrum on a level of real
    spacing h (Sec. 4.1, Eq. polyreq2 and Eq. polyreq3)."""
    t0 = -k * k
    t1 = t0 + 4.0 * dim / (h * np.exp(1j * theta_beta)) ** 2
    t2 = t0 + 4.0 * dim / (h * np.exp(1j * theta_gamma)) ** 2
    return complex(t0), complex(t1), complex(t2)


def basis_ef(t0: complex, t1: complex, t2: complex):
    """e and f of Eq. coefficients_solution: the Vandermonde system of
    Eq. coefficients_system solved for right-hand sides (1, 0, 0) and (1, 1, 1)."""
    rows = [[(x - t0) ** p for p in (1, 2, 3)] for x in (0.0, t1, t2)]
    V = np.array(rows, dtype=np.complex128)
    e = np.linalg.solve(V, np.array([1.0, 0.0, 0.0], dtype=np.complex128))
    f = np.linalg.solve(V, np.array([1.0, 1.0, 1.0], dtype=np.complex128))
    return e, f


def coefficients(e: np.ndarray, f: np.ndarray, phi: float) -> np.ndarray:
    """(c0, c1, c2, c3) of Eq. polynomial: c0 = e^{i phi}, (c1, c2, c3) = e - e^{i phi} f."""
    z = np.exp(1j * phi)
    return np.concatenate([[z], e - z * f])


def evaluate(c: np.ndarray, t0: complex, t) -> np.ndarray:
    """p(t) = c0 + c1 (t - t0) + c2 (t - t0)^2 + c3 (t - t0)^3 (Eq. polynomial)."""
    s = np.asarray(t) - t0
    return c[0] + s * (c[1] + s * (c[2] + s * c[3]))


def first_order(e: np.ndarray, f: np.ndarray, phi, theta_beta: float):
    """First-order stability condition on phi (Eq. firstorder_varphi, sign reading in
    the module docstring): Re(e^{-i phi} c1 e^{-2 i theta_beta}) < 0."""
    z = np.exp(1j * np.asarray(phi))
    c1 = e[0] - z * f[0]
    return np.real(c1 / z * np.exp(-2j * theta_beta)) < 0


def second_order(e: np.ndarray, f: np.ndarray, phi, theta_beta: float):
    """Second-order condition (Eq. secondorder_varphi, as printed)."""
    z = np.exp(1j * np.asarray(phi))
    return 2 * np.real((e[1] / z - f[1]) * np.exp(-4j * theta_beta)) + np.abs(e[0] - z * f[0]) ** 2 < 0


def choose_phi(e: np.ndarray, f: np.ndarray, theta_beta: float) -> Optional[float]:
    """The mapping parameter phi of a level (Sec. 4.5, reading in the module docstring)."""
    fo = first_order(e, f, PHI_GRID, theta_beta)
    ok = fo & second_order(e, f, PHI_GRID, theta_beta)
    if ok.any():
        if ok.all():
            return 0.0
        start = int(np.argmin(ok))           # an infeasible point: arcs do not wrap past it
        r = np.roll(ok, -start)
        best, best_at, run, run_at = 0, 0, 0, 0
        for i, v in enumerate(r):
            if v:
                if run == 0:
                    run_at = i
                run += 1
                if run > best:
                    best, best_at = run, run_at
            else:
                run = 0
        mid = (start + best_at + (best - 1) / 2.0) % len(PHI_GRID)
        return float(np.radians(0.05 * mid))
    if fo.all():
        return 0.0
    return None


def omegas(c: np.ndarray, t0: complex) -> np.ndarray:
    """Weights w_j of the factored form p(t) = prod (1 - w_j t) (Sec. 4.1): the
    reciprocals of p's roots."""
    s_roots = np.roots([c[3], c[2], c[1], c[0]])
    return 1.0 / (s_roots + t0)


def level_polynomial(k: float, h: float, theta_beta: float, theta_gamma: float, dim: int):
    """phi and the Richardson weights of one level, or None if no stable polynomial."""
    t0, t1, t2 = triangle(k, h, theta_beta, theta_gamma, dim)
    e, f = basis_ef(t0, t1, t2)
    phi = choose_phi(e, f, theta_beta)
    if phi is None:
        return None
    return phi, omegas(coefficients(e, f, phi), t0)


def poly_sweep(apply, b: np.ndarray, x: np.ndarray, w: Sequence[complex]) -> np.ndarray:
    """One smoothing step: x <- x + w_j (b - M x) for the three weights (Sec. 4.1)."""
    for wj in w:
        x = x + wj * (b - apply(x))
    return x


def hierarchy_weights(levels: List[Level], k: float, theta_beta: float, theta_gamma: float) -> List:
    """Richardson weights of every smoothed level (all but the coarsest); a level of n
    interior nodes has real spacing 1 / (n + 1)."""
    out = []
    for lev in levels[:-1]:
        lp = level_polynomial(k, 1.0 / (lev.n + 1), theta_beta, theta_gamma, lev.dim)
        if lp is None:
            raise ValueError(f"no stable third-degree polynomial on the level n = {lev.n}")
        out.append(lp[1])
    return out


def vcycle_poly(levels: List[Level], weights: List, b: np.ndarray, nu1: int = 1, nu2: int = 1,
                level: int = 0) -> np.ndarray:
    """x ~ M_l^{-1} b by one V(nu1, nu2) cycle with the polynomial smoother (Sec. 4, the
    same transfers and coarsest solve as the GMRES(s) cycle), zero start."""
    lev = levels[level]
    if level == len(levels) - 1:
        return coarse_solve(lev, b)
    x = np.zeros_like(b, dtype=np.complex128)
    for _ in range(nu1):
        x = poly_sweep(lev.apply, b, x, weights[level])
    r = b - lev.apply(x)
    ec = vcycle_poly(levels, weights, restrict_fw(r), nu1, nu2, level + 1)
    x = x + prolong(ec, lev.n)
    for _ in range(nu2):
        x = poly_sweep(lev.apply, b, x, weights[level])
    return x
