"""Tuned launch choices on the GPU.

- Every launch variant of the 3D TMA-fed Arnoldi and residual passes the autotuner can
  pick (points per thread in y, plane slots in flight, shares of the level), the plain
  passes and their planes per CTA, give a V-cycle that matches the FP64 oracle's point by point (tests/parity_check.py, c64 5e-5) on a
  127^3 heterogeneous problem, whose finest level takes that pass, and 2D tiles-per-CTA
  choices on 255^2 do too.
- helm_autotune on a small problem returns its default and tuned V-cycle times, writes a
  table that helm_tuning_load reads back, and the V-cycle under the tuned choices still
  matches the oracle.
The process's table is restored to the committed one (or emptied) afterwards.
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
    """Load a table of the given entries; restore the committed table afterwards."""
    def load(entries):
        p = tmp_path / "t.json"
        p.write_text(json.dumps({"device": torch.cuda.get_device_name(0), "entries": entries, "runs": []}))
        helm.tuning_load(str(p))
    yield load
    if os.path.exists(COMMITTED):
        helm.tuning_load(COMMITTED)
    else:
        load([])


@pytest.fixture(scope="module")
def cube127():
    w = I.cube_3d(127)
    levels = O.build_hierarchy(3, 127, w.theta_beta, phi=w.phi.astype(np.float64))
    r = I.random_source(3, 127, 77)
    return w, r, O.vcycle(levels, r)


@pytest.mark.parametrize("qy,stages,pieces", [(2, 2, 0), (2, 8, 1), (2, 4, 4), (4, 3, 0), (4, 6, 2), (4, 2, 16)])
def test_tma3_variants_match_oracle(helm, table, cube127, qy, stages, pieces):
    w, r, want = cube127
    entries = [{"pass": "arnoldi", "dim": 3, "P": 128, "prec": 8, "J": J, "v": [1, stages, pieces, qy]}
               for J in (1, 2, 3)]
    entries.append({"pass": "prolong", "dim": 3, "P": 128, "prec": 8, "J": 0, "v": [1, stages, pieces, qy]})
    table(entries)
    assert helm.tuning_get("arnoldi", 3, 128, "c64", 1) == [1, stages, pieces, qy]
    h = helm.Handle(3, 127, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", maxit=1)
    rt = torch.from_numpy(r).cuda().to(torch.complex64)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", "c64"), f"qy={qy} stages={stages} pieces={pieces}")


def test_tma3_off_matches_oracle(helm, table, cube127):
    w, r, want = cube127
    table([{"pass": "arnoldi", "dim": 3, "P": 128, "prec": 8, "J": J, "v": [0, 2, 0, 2]} for J in (1, 2, 3)] +
          [{"pass": "prolong", "dim": 3, "P": 128, "prec": 8, "J": 0, "v": [0, 2, 0, 2]}])
    h = helm.Handle(3, 127, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", maxit=1)
    rt = torch.from_numpy(r).cuda().to(torch.complex64)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", "c64"), "plain 3D pass")


@pytest.mark.parametrize("zc", [2, 8, 16])
def test_3d_plane_counts_match_oracle(helm, table, cube127, zc):
    """The planes per CTA of the plain 3D passes (levels of pitch 64, 32 and 16 of the
    127^3 problem) the autotuner can pick: the V-cycle matches the oracle point by point."""
    w, r, want = cube127
    table([{"pass": "zplanes", "dim": 3, "P": P, "prec": 8, "J": 0, "v": [zc, 0, 0, 0]} for P in (64, 32, 16)])
    assert helm.tuning_get("zplanes", 3, 64, "c64", 0) == [zc, 0, 0, 0]
    h = helm.Handle(3, 127, w.theta_beta, phi=torch.from_numpy(w.phi).cuda(), precision="c64", maxit=1)
    rt = torch.from_numpy(r).cuda().to(torch.complex64)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", "c64"), f"zplanes={zc}")


@pytest.mark.parametrize("tpc", [1, 8])
def test_2d_tiles_per_cta_match_oracle(helm, table, tpc):
    n, k, tb = 255, 40.0, 0.3
    entries = [{"pass": ps, "dim": 2, "P": P, "prec": 8, "J": J, "v": [tpc, 0, 0, 0]}
               for P in (256, 128, 64) for ps, Js in (("arnoldi", (1, 2, 3)), ("restrict", (0,)), ("prolong", (0,)))
               for J in Js]
    table(entries)
    levels = O.build_hierarchy(2, n, tb, k=k)
    r = I.random_source(2, n, 78)
    h = helm.Handle(2, n, tb, k=k, precision="c64", maxit=1)
    rt = torch.from_numpy(r).cuda().to(torch.complex64)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, O.vcycle(levels, r), ("vcycle", "c64"), f"tpc={tpc}")


def test_autotune_writes_a_table_and_keeps_parity(helm, table, tmp_path, cube127):
    table([])
    path = str(tmp_path / "tuned.json")
    w, r, want = cube127
    phi = torch.from_numpy(w.phi).cuda()
    d0, d1 = helm.autotune(3, 127, w.theta_beta, phi=phi, precision="c64", reps=2, path=path)
    assert d0 > 0 and d1 > 0 and d1 <= 1.05 * d0
    d = json.load(open(path))
    assert d["device"] == torch.cuda.get_device_name(0) and d["runs"][-1]["n"] == 127
    helm.tuning_load(path)
    for e in d["entries"]:
        assert helm.tuning_get(e["pass"], e["dim"], e["P"], "c64", e["J"]) == e["v"]
    h = helm.Handle(3, 127, w.theta_beta, phi=phi, precision="c64", maxit=1)
    rt = torch.from_numpy(r).cuda().to(torch.complex64)
    zt = torch.empty_like(rt)
    h.precond_apply(rt, zt)
    assert_parity(zt, want, ("vcycle", "c64"), "after autotune")
