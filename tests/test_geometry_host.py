"""The library's host-side grid geometry (helm_axis_coefficients: the complex map of
Sec. 2, Eq. csggrid, and the three-point coefficients of Eq. csg_dis) against the
oracle's, on the CPU, for layers on both sides (Remark 2.2) and at the far end only
(Benchmark 3 of Sec. 5), on every level size of the hierarchies the tests and the
benchmark run."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def helm():
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


CASES = [(n, w, sides, tg, tb)
         for n in (3, 4, 9, 39, 79, 159, 639, 1023)
         for sides, w in (("both", 0.125), ("both", 1 / 6), ("high", 0.2), ("high", 0.125))
         for tg, tb in ((0.5, 0.3), (np.pi / 6, np.radians(10.3132)), (0.5, 0.0), (0.0, 0.0))]


@pytest.mark.parametrize("n,w,sides,tg,tb", CASES)
def test_axis_coefficients_match_the_oracle(helm, n, w, sides, tg, tb):
    got = helm.axis_coefficients(n, w, tg, tb, sides)
    want = O.coefficients_1d(O.spacings(n, w, tg, tb, sides))
    # the oracle differences the map at the nodes, the library integrates each
    # interval: the oracle's spacings carry a cancellation error of about n ulp
    tol = 5e-16 * (n + 1) + 1e-14
    for g, o in zip(got, want):
        assert np.max(np.abs(g - o)) <= tol * np.max(np.abs(o))


def test_axis_coefficients_reject_bad_arguments(helm):
    for args in ((0, 0.2, 0.5, 0.3, "both"), (15, 0.5, 0.5, 0.3, "both"), (15, 1.0, 0.5, 0.3, "high"),
                 (15, 0.2, 1.6, 0.3, "high"), (15, 0.2, 0.5, -0.1, "both")):
        with pytest.raises(helm.HelmError):
            helm.axis_coefficients(*args)
    with pytest.raises(ValueError):
        helm.axis_coefficients(15, 0.2, 0.5, 0.3, "low")
