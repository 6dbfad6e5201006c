"""The persistent V-cycle segments on the GPU.

The small grid-wide levels of a V-cycle (2D up to 511^2, 3D up to 63^3) can run as one
cooperative launch per half cycle, their passes separated by a grid barrier (switched on
per level through the tuning table; off by default, since the launch-per-pass chain
measured faster on GB300).  Every virtual block does what the block of the ordinary
launch does, so:

- one V-cycle with the persistent segments is bitwise the V-cycle with one launch per
  pass (the segments switched off through the tuning table), in 2D and 3D, complex64
  and complex128, and both match the FP64 oracle point by point;
- a batch of problems of different sizes stays bitwise equal to its solo solves;
- the barrier's bounded wait: with its limit set to zero every waiting CTA gives up at
  once, the launch returns and the solve reports HELM_ETIMEOUT (no trap, no hang); with
  the limit restored a new handle solves correctly.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1012_5379_gb300 import inputs as I
from parity_check import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMITTED = os.path.join(ROOT, "paper_1012_5379_gb300", "tuning.json")


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


@pytest.fixture
def table(helm, tmp_path):
    def load(entries):
        p = tmp_path / "t.json"
        p.write_text(json.dumps({"device": torch.cuda.get_device_name(0), "entries": entries, "runs": []}))
        helm.tuning_load(str(p))
    yield load
    if os.path.exists(COMMITTED):
        helm.tuning_load(COMMITTED)
    else:
        load([])
    helm.set_barrier_timeout(1.0)


def persist_on(dim, prec):
    """Table entries that switch the persistent segments on for every eligible level
    (they are off by default)."""
    sizes = (32, 64, 128, 256, 512) if dim == 2 else (8, 16, 32, 64)
    return [{"pass": "persist", "dim": dim, "P": P, "prec": 8 if prec == "c64" else 16, "J": 0, "v": [1, 0, 0, 0]}
            for P in sizes]


@pytest.mark.parametrize("dim,n,prec", [(2, 511, "c64"), (2, 255, "c128"), (3, 63, "c64"), (3, 63, "c128"),
                                        (3, 127, "c64")])
def test_persistent_vcycle_is_bitwise_the_launch_per_pass_vcycle(helm, table, dim, n, prec):
    k, tb = 0.15 * (n + 1), 0.3
    r = I.random_source(dim, n, 400 + n)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    rt = torch.from_numpy(r).cuda().to(dt)
    outs = {}
    for mode in ("persistent", "per-pass"):
        table(persist_on(dim, prec) if mode == "persistent" else [])
        h = helm.Handle(dim, n, tb, k=k, precision=prec, maxit=1)
        z = torch.empty_like(rt)
        for _ in range(5):   # the first V-cycles run directly, then from the captured graph
            h.precond_apply(rt, z)
        outs[mode] = z.clone()
        h.close()
    assert torch.equal(outs["persistent"], outs["per-pass"])
    levels = O.build_hierarchy(dim, n, tb, k=k)
    assert_parity(outs["persistent"], O.vcycle(levels, r), ("vcycle", prec), "persistent V-cycle")


def test_batch_with_persistent_segments_equals_alone_bitwise(helm, table):
    table(persist_on(2, "c64"))
    ws = I.batch_2d(count=6, seed=93, sizes=(127, 255, 511))
    hs = [helm.Handle(2, w.n, w.theta_beta, k=w.k, precision="c64", restart=w.restart) for w in ws]
    bs = [torch.from_numpy(w.b).cuda() for w in ws]
    xs = [torch.zeros_like(b) for b in bs]
    infos = helm.batch_solve(hs, bs, xs, 1e-6)
    for w, h, b, x, inf in zip(ws, hs, bs, xs, infos):
        solo = torch.zeros_like(b)
        sinfo = h.solve(b, solo, 1e-6)
        assert inf.status == 0 and inf.iters == sinfo.iters and torch.equal(solo, x), w.n


def test_barrier_timeout_reports_etimeout_and_recovers(helm, table):
    table(persist_on(2, "c64"))
    n, k, tb = 255, 30.0, 0.3
    b = torch.from_numpy(I.random_source(2, n, 5)).cuda()
    h = helm.Handle(2, n, tb, k=k, precision="c64", maxit=50)
    x = torch.zeros_like(b)
    helm.set_barrier_timeout(0.0)
    with pytest.raises(helm.HelmError) as e:
        h.solve(b, x, 1e-6)
    assert e.value.code == helm.HELM_ETIMEOUT
    helm.set_barrier_timeout(1.0)
    h.close()   # after HELM_ETIMEOUT the handle's state is invalid; a new one solves correctly
    h = helm.Handle(2, n, tb, k=k, precision="c64", maxit=50)
    x.zero_()
    info = h.solve(b, x, 1e-6)
    assert info.status == 0 and info.rel_res_true <= 1e-6
    levels = O.build_hierarchy(2, n, tb, k=k)
    xs = x.cpu().numpy()
    assert np.linalg.norm(b.cpu().numpy() - levels[0].apply_h(xs)) / np.linalg.norm(b.cpu().numpy()) <= 1.05e-6
    with pytest.raises(helm.HelmError):
        helm.set_barrier_timeout(-1.0)
