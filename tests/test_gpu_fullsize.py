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
- One V-cycle of the 3D 255^3 heterogeneous workload (complex64; its two finest
  levels take the TMA-fed 3D Arnoldi pass) against the oracle's, point by point.
- The 3D heterogeneous solves (FGMRES(40), tol 1e-6) on 127^3 and 255^3: the
  solution's true residual under the oracle's H, and the iteration count within +10%
  (+1) of the oracle's (tests/golden/oracle_iters_cube.json, written by
  tests/golden/make_oracle_iters_cube.py from the oracle alone).
- A batch of 10 problems drawn from the batched workload's sizes {255^2, 511^2,
  1023^2} (more than 8 problems: the batch runs on four stream sets): every result is
  bitwise the problem's solo result, with the same iteration count.
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


def test_vcycle_3d_255_heterogeneous_matches_oracle_c64(helm):
    w = I.cube_3d(255)
    levels = O.build_hierarchy(3, 255, w.theta_beta, phi=w.phi.astype(np.float64))
    src = I.random_source(3, 255, 1005)
    want = O.vcycle(levels, src, 1, 1, 3)
    del levels
    h = helm.Handle(3, 255, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", maxit=1)
    r = torch.from_numpy(src).cuda().to(torch.complex64)
    z = torch.empty_like(r)
    h.precond_apply(r, z)
    h.close()
    assert_parity(z, want, 5e-5, "255^3 V-cycle c64")


def cube_oracle_iters(n):
    path = os.path.join(HERE, "golden", "oracle_iters_cube.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))["by_n"].get(str(n))
    return rec["iters"] if rec else None


def test_solve_3d_127_heterogeneous_iterations(helm):
    ref = cube_oracle_iters(127)
    if ref is None:
        pytest.skip("oracle iteration count of 127^3 not generated")
    w = I.cube_3d(127)
    h = helm.Handle(3, 127, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", restart=40,
                    maxit=400)
    b = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(b)
    info = h.solve(b, x, w.tol)
    h.close()
    assert info.status == 0 and info.rel_res_true <= w.tol
    assert info.iters <= int(1.1 * ref) + 1, (info.iters, ref)
    lev = O.build_hierarchy(3, 127, w.theta_beta, phi=w.phi)[0]
    xs = x.cpu().numpy()
    assert np.linalg.norm(w.b - lev.apply_h(xs)) / np.linalg.norm(w.b) <= 1.05 * w.tol


def test_solve_3d_255_heterogeneous_true_residual(helm):
    w = I.cube_3d(255)
    h = helm.Handle(3, 255, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", restart=40,
                    maxit=400)
    b = torch.from_numpy(w.b).cuda()
    x = torch.zeros_like(b)
    info = h.solve(b, x, w.tol)
    h.close()
    assert info.status == 0 and info.rel_res_true <= w.tol
    ref = cube_oracle_iters(255)
    if ref is not None:
        assert info.iters <= int(1.1 * ref) + 1, (info.iters, ref)
    lev = O.build_hierarchy(3, 255, w.theta_beta, phi=w.phi)[0]
    xs = x.cpu().numpy()
    del x, b
    torch.cuda.empty_cache()
    assert np.linalg.norm(w.b - lev.apply_h(xs)) / np.linalg.norm(w.b) <= 1.05 * w.tol


def test_batch_of_workload_sizes_equals_alone_bitwise(helm):
    ws = I.batch_2d(count=10, seed=91)
    assert {w.n for w in ws} == {255, 511, 1023}
    hs = [helm.Handle(2, w.n, w.theta_beta, k=w.k, precision="c64", restart=w.restart) for w in ws]
    bs = [torch.from_numpy(w.b).cuda() for w in ws]
    xs = [torch.zeros_like(b) for b in bs]
    infos = helm.batch_solve(hs, bs, xs, 1e-6)
    for w, h, b, x, inf in zip(ws, hs, bs, xs, infos):
        solo = torch.zeros_like(b)
        sinfo = h.solve(b, solo, 1e-6)
        assert inf.status == 0 and sinfo.status == 0 and inf.iters == sinfo.iters, (w.n, inf, sinfo)
        assert torch.equal(solo, x), w.n
        assert inf.rel_res_true <= 1e-6
    for h in hs:
        h.close()
