"""Write tests/golden/oracle_iters_1023.json: iteration counts of the FP64 oracle on
the 2D 1023^2 workload (k = 160, unit-variance complex normal source of seed 1001,
ECS layer 1/8 at 0.5 rad, V(1,1) GMRES(3) multigrid down to 3x3, FGMRES without
restart to relative residual 1e-6, Sec. 5) for theta_beta in {0.1, 0.2, 0.3, 0.5}.

Calls only the oracle; takes several minutes of CPU:
    python tests/golden/make_oracle_iters.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import helmholtz as O  # noqa: E402
from paper_1012_5379_gb300 import inputs as I  # noqa: E402

N, K, TOL, SEED = 1023, 160.0, 1e-6, 1001


def main():
    b = I.random_source(2, N, SEED)
    out = {"workload": "2D 1023^2, k=160, random source seed 1001, theta_gamma 0.5, ECS 1/8, V(1,1) GMRES(3), "
                       "FGMRES no restart, tol 1e-6", "by_theta_beta": {}}
    for tb in I.LARGE_2D_BETAS:
        t0 = time.time()
        levels = O.build_hierarchy(2, N, tb, k=K)
        _, info = O.fgmres(levels[0].apply_h, lambda r: O.vcycle(levels, r, 1, 1, 3), b, None, TOL, 0, 300)
        out["by_theta_beta"][str(tb)] = {"iters": info.iters, "restarts": info.restarts,
                                         "rel_res_true": info.rel_res_true, "converged": info.converged}
        print(tb, info.iters, info.restarts, info.rel_res_true, f"{time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters_1023.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
