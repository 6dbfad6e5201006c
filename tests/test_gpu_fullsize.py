"""Parity at the workload sizes the benchmark runs (Sec. 5 setups).

- One V-cycle on the 2D 1023^2 grid (k = 160, theta_beta 0.3, random source) against
  the oracle's V-cycle: the relative 2-norm of the difference and the worst point
  relative to the largest value, each within 5e-5 (c64) or 1e-11 (c128), the
  tolerances of the smaller V-cycle tests (tests/parity_check.py); the same on
  4095^2 (c64), whose finest level takes the TMA-fed pass.
- The four 1023^2 FGMRES solves of the benchmark step (theta_beta 0.1 / 0.2 / 0.3 /
  0.5, complex64 preconditioner, no restart, tol 1e-6): the true residual, recomputed
  with the oracle's H, meets the tolerance, and the iteration count stays within
  +10% (+1) of the oracle's (tests/golden/oracle_iters_1023.json, written by
  tests/golden/make_oracle_iters.py from the oracle alone).
- The 3D 255^3 heterogeneous solve (FGMRES(40), tol 1e-6): the solution's true
  residual under the oracle's H.
"""
import json
import os

import numpy as np
import pytest

from oracle import helmholtz as O
from paper_1012_5379_gb300 import inputs as I
from parity_check import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
N, K = 1023, 160.0


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


@pytest.fixture(scope="module")
def source():
    return I.random_source(2, N, 1001)


@pytest.mark.parametrize("prec,tol", [("c64", 5e-5), ("c128", 1e-11)])
def test_vcycle_1023_matches_oracle(helm, source, prec, tol):
    levels = O.build_hierarchy(2, N, 0.3, k=K)
    want = O.vcycle(levels, source, 1, 1, 3)
    h = helm.Handle(2, N, 0.3, k=K, precision=prec, maxit=1)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    r = torch.from_numpy(source).cuda().to(dt)
    z = torch.empty_like(r)
    h.precond_apply(r, z)
    assert_parity(z, want, tol, f"1023^2 V-cycle {prec}")


def test_vcycle_4095_matches_oracle_c64(helm):
    """The finest level of 4095^2 runs the TMA-fed Arnoldi pass."""
    n, k = 4095, 0.156 * 4096
    src = I.random_source(2, n, 1001)
    levels = O.build_hierarchy(2, n, 0.3, k=k)
    want = O.vcycle(levels, src, 1, 1, 3)
    h = helm.Handle(2, n, 0.3, k=k, precision="c64", maxit=1)
    r = torch.from_numpy(src).cuda().to(torch.complex64)
    z = torch.empty_like(r)
    h.precond_apply(r, z)
    assert_parity(z, want, 5e-5, "4095^2 V-cycle c64")


@pytest.mark.parametrize("tb", [0.1, 0.2, 0.3, 0.5])
def test_solve_1023_iterations_and_residual(helm, source, tb):
    path = os.path.join(HERE, "golden", "oracle_iters_1023.json")
    if not os.path.exists(path):
        pytest.skip("oracle iteration counts not generated")
    ref = json.load(open(path))["by_theta_beta"][str(tb)]
    h = helm.Handle(2, N, tb, k=K, precision="c64", maxit=300)
    b = torch.from_numpy(source).cuda()
    x = torch.zeros_like(b)
    info = h.solve(b, x, 1e-6)
    assert info.status == 0 and info.rel_res_true <= 1e-6
    assert info.iters <= 1.1 * ref["iters"] + 1, (info.iters, ref["iters"])
    lev = O.build_hierarchy(2, N, tb, k=K)[0]
    xs = x.cpu().numpy()
    assert np.linalg.norm(source - lev.apply_h(xs)) / np.linalg.norm(source) <= 1.05e-6


def test_solve_3d_255_heterogeneous_true_residual(helm):
    w = I.cube_3d(255)
    h = helm.Handle(3, 255, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", restart=40,
                    maxit=400)
    b = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(b)
    info = h.solve(b, x, w.tol)
    h.close()
    assert info.status == 0 and info.rel_res_true <= w.tol
    lev = O.build_hierarchy(3, 255, w.theta_beta, phi=w.phi)[0]
    xs = x.cpu().numpy()
    del x, b
    torch.cuda.empty_cache()
    assert np.linalg.norm(w.b - lev.apply_h(xs)) / np.linalg.norm(w.b) <= 1.05 * w.tol
