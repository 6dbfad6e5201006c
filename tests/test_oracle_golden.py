"""Consistency of the stored oracle results the GPU tests compare against.

tests/golden/oracle_iters_1023.json holds the oracle's FGMRES iteration counts on the
2D 1023^2 workload (written by tests/golden/make_oracle_iters.py from the oracle
alone).  Every solve converged to the tolerance in one cycle (no restart is used), and
the counts grow with theta_beta: a larger CSG angle damps less of the Helmholtz
operator's indefiniteness, so the preconditioner is weaker (Sec. 4-5)."""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_iteration_counts_are_consistent():
    rec = json.load(open(os.path.join(HERE, "golden", "oracle_iters_1023.json")))["by_theta_beta"]
    betas = sorted(rec, key=float)
    assert betas == ["0.1", "0.2", "0.3", "0.5"]
    for b in betas:
        assert rec[b]["converged"] and rec[b]["rel_res_true"] <= 1e-6
        assert rec[b]["restarts"] == 1
    iters = [rec[b]["iters"] for b in betas]
    assert iters == sorted(iters) and 20 < iters[0] < iters[-1] < 300
