"""Element-by-element parity of a GPU result against the oracle's.

Two bounds, both relative to the oracle's values `want`:

  * the relative 2-norm of the difference:  ||got - want|| <= tol * ||want||
  * the worst point:    max_p |got_p - want_p| <= tol * max_p |want_p|

The second catches a localized error (one wrong boundary row, a ghost cell, a tile
or TMA box edge, a mis-handled layer interval on a coarse level) that a norm over
10^6 points would dilute by up to three orders of magnitude.

Tolerances by operation and precision (derived from the arithmetic):

  * operator apply: c128 1e-13, c64 1e-6.  5-7 complex terms, each rounded at the
    unit roundoff (1.1e-16 / 6e-8) of the largest coefficient times value, so the
    error of a point is a few units of the largest term, which is bounded by the
    largest output magnitude times the coefficients' ratio (<= 10 on these grids).
  * one V-cycle: c128 1e-11 (different summation order and classical vs modified
    Gram-Schmidt in the smoother, amplified by the cycle's conditioning; measured
    about 1e-15), c64 5e-5 (FP32 through up to 9 levels and about 60 reductions;
    measured 2-5e-7 in the norm).
"""
import numpy as np

TOL = {("op", "c128"): 1e-13, ("op", "c64"): 1e-6,
       ("vcycle", "c128"): 1e-11, ("vcycle", "c64"): 5e-5}


def as_np(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.complex128)


def errors(got, want):
    """(relative 2-norm error, worst-point error relative to the largest value)."""
    g, w = as_np(got), as_np(want)
    assert g.size == w.size, (g.shape, w.shape)
    g, w = g.reshape(-1), w.reshape(-1)
    d = np.abs(g - w)
    return float(np.linalg.norm(g - w) / np.linalg.norm(w)), float(d.max() / np.abs(w).max())


def assert_parity(got, want, tol, what=""):
    """Both bounds at `tol` (a number, or a key of TOL)."""
    if isinstance(tol, tuple):
        tol = TOL[tol]
    e_norm, e_pt = errors(got, want)
    assert np.isfinite(e_norm) and e_norm < tol, f"{what}: relative norm error {e_norm:.3e} >= {tol:.1e}"
    assert np.isfinite(e_pt) and e_pt < tol, f"{what}: worst-point error {e_pt:.3e} (of max |want|) >= {tol:.1e}"
    return e_norm, e_pt
