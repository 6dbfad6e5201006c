"""The library's host-side construction of the polynomial smoother (Sec. 4,
helm_poly_smoother) against the oracle's, on the CPU: the same mapping angle phi (up
to one step of the 0.05 degree grid, where rounding may move an arc's end) and, for
the same phi, the same Richardson weights."""
import numpy as np
import pytest

from oracle import polysmoother as PS


@pytest.fixture(scope="module")
def helm():
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


CASES = [(k, h, tb, d) for d in (2, 3) for k in (5.0, 20.0, 40.0, 100.0) for h in (1 / 256, 1 / 64, 1 / 16, 1 / 4)
         for tb in (np.radians(10.0), np.radians(15.0))]


def test_host_polynomial_matches_the_oracle(helm):
    tg = np.radians(30.0)
    for k, h, tb, d in CASES:
        o = PS.level_polynomial(k, h, tb, tg, d)
        if o is None:
            with pytest.raises(helm.HelmError):
                helm.poly_smoother(k, h, tb, tg, d)
            continue
        phi, w = helm.poly_smoother(k, h, tb, tg, d)
        assert abs(phi - o[0]) <= np.radians(0.05) + 1e-12, (k, h, tb, d)
        t0, t1, t2 = PS.triangle(k, h, tb, tg, d)
        e, f = PS.basis_ef(t0, t1, t2)
        want = np.sort_complex(PS.omegas(PS.coefficients(e, f, phi), t0))
        got = np.sort_complex(np.array(w))
        assert np.max(np.abs(got - want) / np.abs(want)) < 1e-9, (k, h, tb, d)


def test_host_polynomial_rejects_bad_arguments(helm):
    with pytest.raises(helm.HelmError):
        helm.poly_smoother(20.0, 1 / 64, np.radians(35.0), np.radians(30.0), 2)  # theta_beta >= theta_gamma
    with pytest.raises(helm.HelmError):
        helm.poly_smoother(20.0, 0.0, np.radians(10.0), np.radians(30.0), 2)
