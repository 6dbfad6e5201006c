"""Serving (helm_serve_*): continuous batching of solves on one GPU.

Requests submitted while others are on the device are admitted between outer
iterations as the memory budget allows and iterated in the same launches as the
problems already running.  Every result must be bitwise the same as the result of
the same request served alone, and must solve the oracle's ECS operator H (Sec. 2,
Eq. 2.3 with theta_beta = 0) to the requested tolerance.
"""
import time

import numpy as np
import pytest

from oracle import helmholtz as O
from paper_1012_5379_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


def req(i, dim, n, kh):
    return dict(dim=dim, n=n, k=kh * (n + 1), theta_beta=0.3, b=I.random_source(dim, n, 500 + i))


def serve(helm, reqs, stagger=0.0, **kw):
    """Submit `reqs` (optionally `stagger` seconds apart), return solutions, infos, stats."""
    s = helm.Server(**kw)
    try:
        tickets, xs = [], []
        for r in reqs:
            xs.append(np.full_like(r["b"], np.nan))
            tickets.append(s.submit(r["dim"], r["n"], r["k"], r["theta_beta"], r["b"], xs[-1], TOL))
            if stagger:
                time.sleep(stagger)
        out = []
        for x, t in zip(xs, tickets):
            info, lat, rc = s.wait(t, timeout=300.0)
            out.append((x, info, rc, lat))
        stats = s.stats()
    finally:
        s.stop()
    return out, stats


def true_rel_residual(r, x):
    lev = O.build_hierarchy(r["dim"], r["n"], r["theta_beta"], k=r["k"])[0]
    b = r["b"]
    return float(np.linalg.norm(b - lev.apply_h(x)) / np.linalg.norm(b))


MIX = [req(0, 2, 127, 0.2), req(1, 2, 511, 0.15), req(2, 3, 31, 0.25), req(3, 2, 127, 0.3),
       req(4, 2, 255, 0.2), req(5, 3, 15, 0.2), req(6, 2, 1023, 0.1), req(7, 3, 63, 0.2)]


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_served_alone_equals_served_in_mix_bitwise(helm, prec):
    alone = [serve(helm, [r], precision=prec)[0][0] for r in MIX]
    # all at once, and staggered so that requests join problems already iterating
    for stagger in (0.0, 0.002):
        mixed, stats = serve(helm, MIX, stagger=stagger, precision=prec)
        assert stats["completed"] == len(MIX) and stats["peak_active"] >= 2
        for r, (xa, ia, rca, _), (xm, im, rcm, _) in zip(MIX, alone, mixed):
            assert rca == rcm == helm.HELM_OK
            assert ia.iters == im.iters
            assert np.array_equal(xa, xm), (r["dim"], r["n"])
    for r, (x, info, _, lat) in zip(MIX, alone):
        assert info.rel_res_true <= TOL and lat > 0
        if r["n"] <= 255 or r["dim"] == 3:
            assert true_rel_residual(r, x) <= 1.05 * TOL


def test_served_equals_handle_solve(helm):
    r = MIX[0]
    (x, info, rc, _), = serve(helm, [r])[0]
    h = helm.Handle(r["dim"], r["n"], r["theta_beta"], k=r["k"], restart=40, maxit=400)
    xh = np.zeros_like(r["b"])
    ih = h.solve_host(r["b"], xh, TOL)
    assert rc == helm.HELM_OK and ih.iters == info.iters
    assert np.array_equal(x, xh)


def test_budget_limits_admission_and_slots_are_reused(helm):
    reqs = [req(10 + i, 2, 255, 0.1 + 0.05 * i) for i in range(4)]
    one = serve(helm, reqs[:1])[1]["peak_bytes"]
    out, stats = serve(helm, reqs, budget_bytes=int(one * 1.5))
    assert stats["peak_active"] == 1 and stats["peak_bytes"] <= int(one * 1.5)
    assert stats["handles_created"] == 1 and stats["handles_reused"] == 3
    for r, (x, info, rc, _) in zip(reqs, out):
        (xa, ia, _, _), = serve(helm, [r])[0]
        assert rc == helm.HELM_OK and np.array_equal(x, xa)   # re-targeted slot == fresh slot


def test_max_active_caps_concurrency(helm):
    reqs = [req(20 + i, 2, 127, 0.2) for i in range(6)]
    out, stats = serve(helm, reqs, max_active=2)
    assert stats["peak_active"] <= 2 and stats["completed"] == 6
    assert all(rc == helm.HELM_OK for _, _, rc, _ in out)


def test_serving_errors(helm):
    s = helm.Server(budget_bytes=1 << 20)
    try:
        b = I.random_source(2, 100, 1)
        x = np.empty_like(b)
        with pytest.raises(helm.HelmError) as e:
            s.submit(2, 100, 20.0, 0.3, b, x, TOL)            # n + 1 not a power of two
        assert e.value.code == helm.HELM_EINVAL
        with pytest.raises(helm.HelmError):
            s.submit(4, 127, 20.0, 0.3, b, x, TOL)            # dimension
        b = I.random_source(2, 511, 1)
        x = np.empty_like(b)
        t = s.submit(2, 511, 60.0, 0.3, b, x, TOL)            # cannot fit 1 MiB
        info, lat, rc = s.wait(t, timeout=60.0)
        assert rc == helm.HELM_ENOMEM and s.stats()["rejected"] == 1
        with pytest.raises(helm.HelmError):
            s.poll(t)                                          # ticket released
    finally:
        s.stop()
    s = helm.Server()
    try:
        b = I.random_source(2, 1023, 2)
        x = np.empty_like(b)
        t = s.submit(2, 1023, 102.4, 0.3, b, x, TOL)
        with pytest.raises(helm.HelmError) as e:
            s.wait(t, timeout=0.0)
        assert e.value.code == helm.HELM_ETIMEOUT
        info, lat, rc = s.wait(t, timeout=120.0)
        assert rc == helm.HELM_OK and info.rel_res_true <= TOL
    finally:
        s.stop()


def test_stop_drains_pending_requests(helm):
    s = helm.Server()
    reqs = [req(40 + i, 2, 255, 0.15) for i in range(5)]
    xs = [np.full_like(r["b"], np.nan) for r in reqs]
    for r, x in zip(reqs, xs):
        s.submit(2, 255, r["k"], 0.3, r["b"], x, TOL)
    s.stop()   # returns once every admitted and queued request has finished
    assert all(np.isfinite(x).all() for x in xs)
    assert true_rel_residual(reqs[-1], xs[-1]) <= 1.05 * TOL


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_source_is_retired_with_enumeric(helm, bad):
    """A request whose source holds a NaN or an Inf (injected on the host) is retired
    with HELM_ENUMERIC; requests served beside it are unaffected (bitwise equal to
    being served alone)."""
    good = req(60, 2, 127, 0.2)
    badr = dict(req(61, 2, 127, 0.2))
    badr["b"] = badr["b"].copy()
    badr["b"][17, 40] = bad
    out, stats = serve(helm, [badr, good])
    (xb, ib, rcb, _), (xg, ig, rcg, _) = out
    assert rcb == helm.HELM_ENUMERIC and ib.status == helm.HELM_ENUMERIC
    assert rcg == helm.HELM_OK and ig.rel_res_true <= TOL
    (xa, ia, _, _), = serve(helm, [good])[0]
    assert ia.iters == ig.iters and np.array_equal(xa, xg)
