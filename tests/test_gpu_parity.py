"""GPU parity tests: the CUDA path through the C ABI against the FP64 oracle.

Every element-wise comparison bounds both the relative 2-norm of the difference and
the worst point relative to the largest value (tests/parity_check.py), at:
  * operator apply:  c128 1e-13, c64 1e-6 (5-7 complex terms, FP32 rounding ~6e-8
    each, cancellation bounded by the coefficient magnitudes)
  * one V-cycle:     c128 1e-11 (different summation order and CGS vs MGS in the
    smoother; measured ~1e-15), c64 5e-5 (FP32 arithmetic through ~9 levels and 60+
    reductions; measured ~5e-7)
  * FGMRES solve:    true residual <= tol recomputed by the oracle's H; iterations
    within +10% (+1) of the oracle's; solution within a few tol of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from parity_check import assert_parity
from paper_1012_5379_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TG, WF = I.THETA_GAMMA, I.ECS_FRAC


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


def dev(a, prec="c128"):
    t = torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return t.to(torch.complex64) if prec == "c64" else t


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("dim,n,prec,field", [(2, 31, "c128", False), (2, 47, "c64", False),
                                              (3, 15, "c128", True), (3, 15, "c64", True),
                                              (2, 63, "c128", True)])
def test_operator_apply(helm, dim, n, prec, field):
    tb, k = 0.35, 11.0
    phi = None
    if field:
        phi = I.bump_field(n, 5, k0=k) if dim == 3 else \
            np.random.default_rng(3).uniform(50, 300, (n, n)).astype(np.float32)
    levels = O.build_hierarchy(dim, n, tb, TG, WF, k=None if field else k,
                               phi=phi.astype(np.float64) if field else None)
    h = helm.Handle(dim, n, tb, k=None if field else k,
                    phi=torch.from_numpy(phi).cuda() if field else None, precision=prec)
    v = I.random_source(dim, n, 3)
    tol = 1e-13 if prec == "c128" else 1e-6
    for which in "MH":
        want = levels[0].apply(v) if which == "M" else levels[0].apply_h(v)
        vt = dev(v, prec)
        wt = torch.empty_like(vt)
        h.apply_operator(vt, wt, which)
        assert_parity(wt, want, tol, which)


# ------------------------------------------------------------------ complex shifted Laplacian variant
@pytest.mark.parametrize("dim,n,prec,tb,eps", [(2, 63, "c128", 0.0, 0.5), (3, 15, "c128", 0.0, 0.5),
                                               (2, 127, "c64", 0.0, 0.5), (2, 63, "c128", 0.2, 0.25)])
def test_csl_operator_and_vcycle(helm, dim, n, prec, tb, eps):
    """M = L - (1 + i eps) k^2: the CSL shift alone (theta_beta = 0) or combined with
    the stretched grid; the operators and one V-cycle against the oracle's."""
    k = 0.15 * (n + 1)
    levels = O.build_hierarchy(dim, n, tb, TG, WF, k=k, csl_eps=eps)
    h = helm.Handle(dim, n, tb, k=k, precision=prec, csl_eps=eps)
    v = I.random_source(dim, n, 7)
    for which in "MH":
        want = levels[0].apply(v) if which == "M" else levels[0].apply_h(v)
        vt = dev(v, prec)
        wt = torch.empty_like(vt)
        h.apply_operator(vt, wt, which)
        assert_parity(wt, want, ("op", prec), which)
    want = O.vcycle(levels, v)
    vt = dev(v, prec)
    zt = torch.empty_like(vt)
    h.precond_apply(vt, zt)
    assert_parity(zt, want, ("vcycle", prec), "V-cycle")


def test_csl_solve(helm):
    """FGMRES preconditioned by the CSL V-cycle (theta_beta = 0, eps = 0.5) on 127^2,
    k = 20: true residual under the oracle's H, iterations within +10% (+1)."""
    n, k, eps, tol = 127, 20.0, 0.5, 1e-6
    b = I.random_source(2, n, 33)
    levels = O.build_hierarchy(2, n, 0.0, TG, WF, k=k, csl_eps=eps)
    _, io = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=tol, restart=0, maxit=200)
    h = helm.Handle(2, n, 0.0, k=k, precision="c64", csl_eps=eps)
    bt = dev(b)
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, tol)
    x = xt.cpu().numpy()
    assert info.status == 0
    assert np.linalg.norm(b - levels[0].apply_h(x)) / np.linalg.norm(b) <= tol * 1.0001
    assert info.iters <= int(1.1 * io.iters) + 1


def test_csl_argument_checks(helm):
    """A negative or non-finite shift, or a shift with a k field, is refused."""
    for bad in (-0.1, float("nan")):
        with pytest.raises(helm.HelmError):
            helm.Handle(2, 31, 0.0, k=5.0, csl_eps=bad)
    phi = torch.full((31, 31), 25.0, dtype=torch.float32, device="cuda")
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 31, 0.0, phi=phi, csl_eps=0.5)


# ------------------------------------------------------------------ polynomial smoother (Sec. 4)
def poly_weights(helm, levels, k, tb, tg):
    """The oracle's Richardson weights, for the library's choice of phi on every
    smoothed level (the two choose it by the same rule; a grid step apart at most), in
    the library's order (real part, then imaginary part)."""
    from oracle import polysmoother as PS
    out = []
    for lev in levels[:-1]:
        h = 1.0 / (lev.n + 1)
        phi, _ = helm.poly_smoother(k, h, tb, tg, lev.dim)
        t0, t1, t2 = PS.triangle(k, h, tb, tg, lev.dim)
        e, f = PS.basis_ef(t0, t1, t2)
        out.append(sorted(PS.omegas(PS.coefficients(e, f, phi), t0), key=lambda c: (c.real, c.imag)))
    return out


@pytest.mark.parametrize("dim,n,prec,nu1,nu2", [(2, 63, "c128", 1, 1), (2, 127, "c128", 2, 1), (3, 15, "c128", 1, 1),
                                                (2, 255, "c64", 1, 1), (3, 31, "c64", 1, 2)])
def test_poly_vcycle_matches_oracle(helm, dim, n, prec, nu1, nu2):
    """One V-cycle with the third-degree polynomial smoother (theta_beta = 10,
    theta_gamma = 30 degrees) against the oracle's."""
    from oracle import polysmoother as PS
    k, tb, tg = 0.1 * (n + 1), np.radians(10.0), np.radians(30.0)
    levels = O.build_hierarchy(dim, n, tb, tg, WF, k=k)
    r = I.random_source(dim, n, 40 + n)
    want = PS.vcycle_poly(levels, poly_weights(helm, levels, k, tb, tg), r, nu1, nu2)
    h = helm.Handle(dim, n, tb, k=k, theta_gamma=tg, precision=prec, nu1=nu1, nu2=nu2, smoother="poly")
    rt = dev(r, prec)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, 1e-11 if prec == "c128" else 1e-4, "polynomial V-cycle")


def test_poly_solve(helm):
    """FGMRES preconditioned by the polynomial-smoothed V-cycle on 127^2, k = 20,
    theta_beta = 10 degrees: true residual under the oracle's H, iterations within +10%
    (+1) of the oracle's."""
    from oracle import polysmoother as PS
    n, k, tb, tg, tol = 127, 20.0, np.radians(10.0), TG, 1e-6
    b = I.random_source(2, n, 33)
    levels = O.build_hierarchy(2, n, tb, tg, WF, k=k)
    w = poly_weights(helm, levels, k, tb, tg)
    _, io = O.fgmres(levels[0].apply_h, lambda v: PS.vcycle_poly(levels, w, v), b, tol=tol, restart=0, maxit=300)
    h = helm.Handle(2, n, tb, k=k, theta_gamma=tg, precision="c64", smoother="poly")
    bt = dev(b)
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, tol)
    x = xt.cpu().numpy()
    assert info.status == 0
    assert np.linalg.norm(b - levels[0].apply_h(x)) / np.linalg.norm(b) <= tol * 1.0001
    assert info.iters <= int(1.1 * io.iters) + 1


def test_poly_argument_checks(helm):
    """No stable polynomial (theta_beta too small), a k field or a complex shift:
    refused."""
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 127, np.radians(1.0), k=60.0, theta_gamma=np.radians(30.0), smoother="poly")
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 31, 0.2, k=5.0, csl_eps=0.5, smoother="poly")
    phi = torch.full((31, 31), 25.0, dtype=torch.float32, device="cuda")
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 31, 0.2, phi=phi, smoother="poly")


# ------------------------------------------------------------------ one V-cycle
VC_CASES = [
    (2, 15, "c128"), (2, 31, "c128"), (2, 63, "c128"), (2, 127, "c128"), (2, 255, "c128"),
    (3, 7, "c128"), (3, 15, "c128"), (3, 31, "c128"),
    (2, 63, "c64"), (2, 255, "c64"), (2, 511, "c64"), (3, 31, "c64"), (3, 63, "c64"), (3, 127, "c64"),
]


@pytest.mark.parametrize("dim,n,prec", VC_CASES)
def test_vcycle_matches_oracle(helm, dim, n, prec):
    k, tb = 0.15 * (n + 1), 0.3
    levels = O.build_hierarchy(dim, n, tb, TG, WF, k=k)
    r = I.random_source(dim, n, 100 + n)
    want = O.vcycle(levels, r)
    h = helm.Handle(dim, n, tb, k=k, precision=prec)
    rt = dev(r, prec)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", prec), "V-cycle")


@pytest.mark.parametrize("nu1,nu2,s", [(1, 0, 3), (2, 1, 3), (1, 1, 2), (1, 1, 4), (0, 1, 3), (2, 2, 1)])
def test_vcycle_variants(helm, nu1, nu2, s):
    """V(nu1, nu2) with GMRES(s), the paper's Table 1 family."""
    n, k, tb = 127, 20.0, 0.18
    levels = O.build_hierarchy(2, n, tb, np.pi / 6, WF, k=k)
    r = I.random_source(2, n, 5)
    want = O.vcycle(levels, r, nu1, nu2, s)
    h = helm.Handle(2, n, tb, k=k, theta_gamma=np.pi / 6, precision="c128", nu1=nu1, nu2=nu2, s=s)
    rt = dev(r)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, 1e-11, "V-cycle")


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_vcycle_heterogeneous_3d(helm, prec):
    n = 31
    phi = I.bump_field(n, 1002, k0=0.3 * (n + 1))
    levels = O.build_hierarchy(3, n, 0.4, TG, WF, phi=phi.astype(np.float64))
    r = I.random_source(3, n, 8)
    want = O.vcycle(levels, r)
    h = helm.Handle(3, n, 0.4, phi=torch.from_numpy(phi).cuda(), precision=prec)
    rt = dev(r, prec)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", prec), "V-cycle")


@pytest.mark.parametrize("dim,n,prec", [(2, 255, "c128"), (2, 255, "c64"), (3, 31, "c64"), (3, 15, "c128")])
def test_vcycle_straddling_layer(helm, dim, n, prec):
    """A layer of width 0.1, which no dyadic spacing divides: on every level the
    interval holding the turning point is part layer, part interior (exact segment
    integrals of the map, Sec. 2), so every grid-wide level has mixed spacings near
    each face.  Operator and one V-cycle, point by point."""
    k, tb, wf = 0.15 * (n + 1), 0.3, 0.1
    levels = O.build_hierarchy(dim, n, tb, TG, wf, k=k)
    h = helm.Handle(dim, n, tb, k=k, precision=prec, ecs_frac=wf)
    r = I.random_source(dim, n, 300 + n)
    for which in "MH":
        want = levels[0].apply(r) if which == "M" else levels[0].apply_h(r)
        rt = dev(r, prec)
        wt = torch.empty_like(rt)
        h.apply_operator(rt, wt, which)
        assert_parity(wt, want, ("op", prec), which)
    want = O.vcycle(levels, r)
    rt = dev(r, prec)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", prec), "V-cycle")


def test_vcycle_input_precisions_and_edge_cases(helm):
    n = 63
    h = helm.Handle(2, n, 0.3, k=10.0, precision="c64")
    # zero input -> zero output (empty sweeps everywhere)
    z0 = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    out = torch.full_like(z0, 1 + 1j)
    h.precond_apply(z0, out)
    assert torch.count_nonzero(out).item() == 0
    # complex128 in/out on a complex64 handle equals complex64 in/out
    r = I.random_source(2, n, 2)
    a = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    h.precond_apply(dev(r), a)
    b = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    h.precond_apply(dev(r, "c64"), b)
    assert_parity(a, b, 1e-6, "c128 vs c64 input")
    # scaling: V(alpha r) = alpha V(r) up to rounding (GMRES is scale-equivariant)
    c = torch.empty_like(a)
    h.precond_apply(dev(1e3 * r), c)
    assert_parity(c.cpu().numpy() / 1e3, a, 1e-5, "scaled input")


def test_invalid_arguments(helm):
    with pytest.raises(helm.HelmError) as e:
        helm.Handle(4, 15, 0.3, k=1.0)
    assert e.value.code == helm.HELM_EINVAL
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 15, 2.0, k=1.0)   # theta_beta >= pi/2
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 15, 0.3, k=1.0, s=5)
    with pytest.raises(helm.HelmError):
        helm.Handle(2, 16, 0.3, k=1.0)   # n + 1 odd: the 16^2 coarsest grid is too large
    h = helm.Handle(2, 15, 0.3, k=1.0)
    b = torch.zeros((15, 15), dtype=torch.complex128, device="cuda")
    with pytest.raises(helm.HelmError):
        h.solve(b, torch.zeros_like(b), -1.0)


# ------------------------------------------------------------------ FGMRES solves
def oracle_solve(dim, n, tb, k, b, tol, restart=0, phi=None):
    levels = O.build_hierarchy(dim, n, tb, TG, WF, k=k, phi=phi)
    x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=tol, restart=restart)
    return levels, x, info


@pytest.mark.parametrize("prec,tol", [("c128", 1e-8), ("c64", 1e-6), ("c64", 1e-8)])
def test_solve_small_2d(helm, prec, tol):
    """The small configuration: 127^2, k = 20, point source, theta_beta = 0.4."""
    w = I.small_2d()
    levels, xo, io = oracle_solve(2, w.n, w.theta_beta, w.k, w.b, tol)
    h = helm.Handle(2, w.n, w.theta_beta, k=w.k, precision=prec)
    bt = dev(w.b)
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, tol)
    x = xt.cpu().numpy()
    true = np.linalg.norm(w.b - levels[0].apply_h(x)) / np.linalg.norm(w.b)
    assert info.status == 0 and true <= tol * 1.0001
    assert abs(info.rel_res_true - true) <= 1e-3 * true + 1e-15
    assert info.iters <= int(1.1 * io.iters) + 1
    assert rel(x, xo) < 50 * tol


@pytest.mark.parametrize("restart", [5, 12])
def test_solve_restarted(helm, restart):
    n, k, tb = 63, 25.0, 0.3
    b = I.random_source(2, n, 21)
    levels, xo, io = oracle_solve(2, n, tb, k, b, 1e-7, restart=restart)
    h = helm.Handle(2, n, tb, k=k, precision="c128", restart=restart)
    bt = dev(b)
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, 1e-7)
    assert info.status == 0 and info.restarts >= 2
    assert abs(info.iters - io.iters) <= max(1, int(0.1 * io.iters))


def test_solve_initial_guess_and_zero_rhs(helm):
    n, k, tb = 63, 15.0, 0.3
    b = I.random_source(2, n, 4)
    levels, xo, _ = oracle_solve(2, n, tb, k, b, 1e-10)
    h = helm.Handle(2, n, tb, k=k, precision="c128")
    bt = dev(b)
    # exact initial guess: zero iterations
    xt = dev(xo)
    info = h.solve(bt, xt, 1e-8)
    assert info.iters == 0 and info.status == 0
    # zero right-hand side: x = 0, no iterations
    zb = torch.zeros_like(bt)
    xz = torch.ones_like(bt)
    info = h.solve(zb, xz, 1e-8)
    assert info.iters == 0 and torch.count_nonzero(xz).item() == 0


def test_solve_maxit_reports_noconv(helm):
    n = 63
    h = helm.Handle(2, n, 0.3, k=25.0, precision="c64", maxit=3)
    bt = dev(I.random_source(2, n, 1))
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, 1e-12)
    assert info.status == helm.HELM_ENOCONV and info.iters == 3


def test_solve_3d_heterogeneous(helm):
    n = 31
    phi = I.bump_field(n, 1002, k0=0.3 * (n + 1))
    b = I.point_source(3, n)
    levels, xo, io = oracle_solve(3, n, 0.4, None, b, 1e-6, restart=40, phi=phi.astype(np.float64))
    h = helm.Handle(3, n, 0.4, phi=torch.from_numpy(phi).cuda(), precision="c64", restart=40)
    bt = dev(b)
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, 1e-6)
    x = xt.cpu().numpy()
    true = np.linalg.norm(b - levels[0].apply_h(x)) / np.linalg.norm(b)
    assert info.status == 0 and true <= 1e-6
    assert info.iters <= int(1.1 * io.iters) + 1


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_source_reports_enumeric(helm, bad):
    """A NaN or an Inf in the source (injected on the host) ends helm_solve with
    HELM_ENUMERIC before any V-cycle; in a batch only that problem fails, and the other
    one's result is bitwise its solo result."""
    n = 63
    b = I.random_source(2, n, 9)
    bb = b.copy()
    bb[5, 7] = bad
    h = helm.Handle(2, n, 0.3, k=10.0, precision="c64")
    x = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    info = h.solve(dev(bb), x, 1e-6)
    assert info.status == helm.HELM_ENUMERIC and info.iters == 0
    h2 = helm.Handle(2, n, 0.3, k=12.0, precision="c64")
    xs = [torch.zeros_like(x), torch.zeros_like(x)]
    infos = helm.batch_solve([h, h2], [dev(bb), dev(b)], xs, 1e-6)
    assert infos[0].status == helm.HELM_ENUMERIC and infos[1].status == helm.HELM_OK
    solo = torch.zeros_like(x)
    sinfo = h2.solve(dev(b), solo, 1e-6)
    assert sinfo.iters == infos[1].iters and torch.equal(solo, xs[1])


def test_solve_host_buffers(helm):
    w = I.small_2d()
    h = helm.Handle(2, w.n, w.theta_beta, k=w.k, precision="c64")
    x = np.zeros_like(w.b)
    info = h.solve_host(w.b, x, 1e-6)
    levels = O.build_hierarchy(2, w.n, w.theta_beta, TG, WF, k=w.k)
    assert info.status == 0
    assert np.linalg.norm(w.b - levels[0].apply_h(x)) / np.linalg.norm(w.b) <= 1e-6


# ------------------------------------------------------------------ batching
def test_batch_equals_alone_bitwise(helm):
    """Mixed sizes in one batch: every result is bitwise the one of its solo solve
    (per-problem reductions in a fixed order)."""
    ws = I.batch_2d(count=5, seed=77, sizes=(63, 127, 255))
    hs, bs, xs = [], [], []
    for w in ws:
        hs.append(helm.Handle(2, w.n, w.theta_beta, k=w.k, precision="c64", restart=w.restart))
        bs.append(dev(w.b))
        xs.append(torch.zeros_like(bs[-1]))
    infos = helm.batch_solve(hs, bs, xs, 1e-6)
    for w, h, b, x, inf in zip(ws, hs, bs, xs, infos):
        solo = torch.zeros_like(b)
        sinfo = h.solve(b, solo, 1e-6)
        assert inf.status == 0 and inf.iters == sinfo.iters
        assert torch.equal(solo, x)
        levels = O.build_hierarchy(2, w.n, w.theta_beta, TG, WF, k=w.k)
        xn = x.cpu().numpy()
        assert np.linalg.norm(w.b - levels[0].apply_h(xn)) / np.linalg.norm(w.b) <= 1e-6
