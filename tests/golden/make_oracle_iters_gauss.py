"""Write tests/golden/oracle_iters_gauss.json: iteration counts of the FP64 oracle on
the Gaussian model (Benchmark 3 of Sec. 5, ``inputs.gaussian_model``: the five
(k, grid) columns of Tables 4 and 5 for nu = 1 and nu = 7, V(1,0) and V(1,1) cycles
with GMRES(3) smoothing, FGMRES without restart to relative residual 1e-7).

Calls only the oracle; takes about half an hour of CPU (the 512^2 columns dominate):
    python tests/golden/make_oracle_iters_gauss.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import helmholtz as O  # noqa: E402
from paper_1012_5379_gb300 import inputs as I  # noqa: E402


def key(nu, k, nint, cycle):
    return f"nu={nu:g} k={k:g} nint={nint} V({cycle})"


def main():
    out = {"workload": "Gaussian model (Sec. 5, Benchmark 3), inputs.gaussian_model; GMRES(3) smoothing, "
                       "FGMRES no restart, tol 1e-7", "iters": {}}
    for nu in (1.0, 7.0):
        for k, nint in I.GAUSS_COLUMNS:
            w = I.gaussian_model(nint, k, nu)
            levels = O.build_hierarchy(2, w.n, w.theta_beta, w.theta_gamma, w.ecs_frac,
                                       phi=w.phi.astype(np.float64), ecs_sides="high")
            for cycle in ("1,0", "1,1"):
                nu1, nu2 = map(int, cycle.split(","))
                t0 = time.time()
                _, info = O.fgmres(levels[0].apply_h, lambda r: O.vcycle(levels, r, nu1, nu2, 3), w.b, None,
                                   w.tol, 0, 600)
                out["iters"][key(nu, k, nint, cycle)] = {"iters": info.iters, "rel_res_true": info.rel_res_true,
                                                          "converged": info.converged}
                print(key(nu, k, nint, cycle), info.iters, info.rel_res_true, f"{time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters_gauss.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
