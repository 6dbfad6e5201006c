"""Short restart lengths of the outer FGMRES (Sec. 5) against the oracle.

The outer passes share one partial-sum buffer; the multi-dot's group counters, which
must read zero at every call, used to sit at its end, where the other passes' partials
overwrote them when the basis was short (restart or maxit of a few vectors): the inner
products came out wrong and the solve made no progress (true residual 1.0 after four
iterations on 63^3).  These solves end at maxit, after a cycle end (restart = maxit)
or after several restarts, and are compared with the oracle's FGMRES run for the same
number of iterations: the final true residual within 1% of the oracle's and the
solution within 1e-3 (relative 2-norm; the complex64 V-cycle perturbs each
preconditioned vector by about 1e-6, and FGMRES carries that into x), in both basis
arithmetics.
"""
import numpy as np
import pytest

from oracle import helmholtz as O
from paper_1012_5379_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


CASES = [(3, 63, 4, 4), (3, 63, 8, 8), (3, 63, 12, 4), (2, 255, 4, 4), (2, 255, 12, 3)]


@pytest.fixture(scope="module")
def oracle_runs():
    out = {}
    for dim, n, maxit, restart in CASES:
        k = 0.156 * (n + 1)
        levels = O.build_hierarchy(dim, n, 0.3, k=k)
        b = I.random_source(dim, n, 1001)
        x, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), b, tol=1e-12, restart=restart,
                           maxit=maxit)
        out[(dim, n, maxit, restart)] = (b, x, info)
    return out


@pytest.mark.parametrize("dim,n,maxit,restart", CASES)
@pytest.mark.parametrize("basis", ["f64", "df"])
def test_short_restart_matches_oracle(helm, oracle_runs, dim, n, maxit, restart, basis):
    b, xo, io = oracle_runs[(dim, n, maxit, restart)]
    h = helm.Handle(dim, n, 0.3, k=0.156 * (n + 1), precision="c64", restart=restart, maxit=maxit, basis=basis)
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    info = h.solve(bt, xt, 1e-12)
    assert info.status == helm.HELM_ENOCONV and info.iters == maxit == io.iters
    assert info.basis == basis
    assert abs(info.rel_res_true - io.rel_res_true) <= 0.01 * io.rel_res_true, (info.rel_res_true, io.rel_res_true)
    x = xt.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-3 * np.linalg.norm(xo)
