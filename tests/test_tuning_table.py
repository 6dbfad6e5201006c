"""CPU checks of the tuned launch-choice table (no GPU): helm_tuning_load reads a JSON
table and helm_tuning_get returns each entry by (pass, dimension, level pitch,
precision, Arnoldi step), nothing for absent keys (the built-in defaults apply); a
malformed or missing file is refused and leaves the current table; the committed table
beside the library parses."""
import json
import os

import pytest

from paper_1012_5379_gb300 import helm as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_1012_5379_gb300", "tuning.json")


@pytest.fixture(scope="module")
def lib():
    from paper_1012_5379_gb300 import build
    build.build()
    try:
        return H.load()
    except OSError as e:  # pragma: no cover - needs libcudart on the loader path
        pytest.skip(f"libhelm.so does not load here: {e}")


def write(tmp_path, entries, device="", name="t.json"):
    p = tmp_path / name
    p.write_text(json.dumps({"device": device, "entries": entries, "runs": [{"note": "x"}]}))
    return str(p)


def test_lookup_of_loaded_entries(lib, tmp_path):
    path = write(tmp_path, [
        {"pass": "arnoldi", "dim": 3, "P": 256, "prec": 8, "J": 2, "v": [1, 6, 0, 0]},
        {"pass": "arnoldi", "dim": 3, "P": 256, "prec": 8, "J": 3, "v": [0, 2, 0, 0]},
        {"pass": "restrict", "dim": 2, "P": 1024, "prec": 8, "J": 0, "v": [4, 0, 0, 0]},
        {"pass": "prolong", "dim": 2, "P": 1024, "prec": 16, "J": 0, "v": [2, 0, 0, 0]},
    ])
    H.tuning_load(path)
    assert H.tuning_get("arnoldi", 3, 256, "c64", 2) == [1, 6, 0, 0]
    assert H.tuning_get("arnoldi", 3, 256, "c64", 3) == [0, 2, 0, 0]
    assert H.tuning_get("restrict", 2, 1024, "c64") == [4, 0, 0, 0]
    assert H.tuning_get("prolong", 2, 1024, "c128") == [2, 0, 0, 0]
    # absent keys: another step, pitch, precision or pass
    assert H.tuning_get("arnoldi", 3, 256, "c64", 1) is None
    assert H.tuning_get("arnoldi", 3, 128, "c64", 2) is None
    assert H.tuning_get("prolong", 2, 1024, "c64") is None
    assert H.tuning_get("arnoldi", 2, 1024, "c64", 0) is None


def test_malformed_or_missing_tables_are_refused(lib, tmp_path):
    good = write(tmp_path, [{"pass": "restrict", "dim": 2, "P": 512, "prec": 8, "J": 0, "v": [8, 0, 0, 0]}])
    H.tuning_load(good)
    bad = tmp_path / "bad.json"
    bad.write_text('{"device": "x", "entries": [{"pass": "restrict", "dim": 2')
    with pytest.raises(H.HelmError):
        H.tuning_load(str(bad))
    with pytest.raises(H.HelmError):
        H.tuning_load(str(tmp_path / "absent.json"))
    unknown = write(tmp_path, [{"pass": "smooth", "dim": 2, "P": 512, "prec": 8, "J": 0, "v": [1]}], name="u.json")
    with pytest.raises(H.HelmError):
        H.tuning_load(unknown)
    assert H.tuning_get("restrict", 2, 512, "c64") == [8, 0, 0, 0]   # the good table stayed
    with pytest.raises(H.HelmError):
        H.tuning_get("smooth", 2, 512, "c64")


def test_committed_table_parses(lib):
    if not os.path.exists(TABLE):
        pytest.skip("no committed tuning table")
    d = json.load(open(TABLE))
    H.tuning_load(TABLE)
    for e in d["entries"]:
        prec = "c64" if e["prec"] == 8 else "c128"
        assert H.tuning_get(e["pass"], e["dim"], e["P"], prec, e["J"]) == e["v"]
    for r in d["runs"]:
        assert r["tuned_ms_per_vcycle"] <= r["default_ms_per_vcycle"] * 1.05
