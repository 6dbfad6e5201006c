"""Write tests/golden/oracle_iters_cube.json: the FP64 oracle's FGMRES(40) iteration
count on the 3D heterogeneous workload (unit cube, n^3 interior nodes, k(x) =
80 (1 + 0.3 g(x)) with 8 seeded Gaussian bumps of width 0.1, point source at the
centre, theta_beta 0.4, ECS layer 1/8 at 0.5 rad, V(1,1) GMRES(3) multigrid down to
3^3, relative residual 1e-6; Sec. 5's solver in 3D) for n = 127 and n = 255.

Calls only the oracle.  The 255^3 solve takes about half an hour of one CPU core and
about 25 GB of memory (the FGMRES(40) bases V and Z in complex128):
    python tests/golden/make_oracle_iters_cube.py [127] [255]
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

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters_cube.json")


def main(sizes):
    out = json.load(open(PATH)) if os.path.exists(PATH) else {
        "workload": "3D unit cube, k(x)=80(1+0.3 g(x)), 8 bumps (seed 1002, sigma 0.1), point source, "
                    "theta_beta 0.4, theta_gamma 0.5, ECS 1/8, V(1,1) GMRES(3), FGMRES(40), tol 1e-6",
        "by_n": {}}
    for n in sizes:
        w = I.cube_3d(n)
        t0 = time.time()
        levels = O.build_hierarchy(3, n, w.theta_beta, I.THETA_GAMMA, I.ECS_FRAC, phi=w.phi.astype(np.float64))
        _, info = O.fgmres(levels[0].apply_h, lambda r: O.vcycle(levels, r, 1, 1, 3), w.b, None, w.tol,
                           w.restart, 400)
        out["by_n"][str(n)] = {"iters": info.iters, "restarts": info.restarts,
                               "rel_res_true": info.rel_res_true, "converged": info.converged}
        print(n, info.iters, info.restarts, info.rel_res_true, f"{time.time() - t0:.0f}s", flush=True)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [127, 255])
