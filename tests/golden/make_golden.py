"""Writes tests/golden/grf256_steady.json with the FP64 oracle only.

The 256^3 tortuosity workload (thresholded Gaussian random field, porosity
0.35, c = 1 / c = 0 held on the x faces, D = 1) is solved to its discrete
steady state by the oracle's conjugate-gradient solver (relative residual
1e-13), and the script stores D_eff, tau, psi, the two face fluxes and the
steady values at 4096 seeded sample voxels.  The GPU test compares its own
steady state against these numbers.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import grf256  # noqa: E402


def main():
    t0 = time.time()
    phi, u0, phys = grf256()
    P = oracle.Problem(phi, phys)
    u, rel, iters = P.steady_cg(u0, tol=1e-13, maxit=200000)
    red = P.reduce(u)[0]
    d_eff, tau, psi = P.effective_D(u)
    rng = np.random.default_rng(4242)
    act = np.argwhere(P.active > 0)
    pick = act[rng.choice(len(act), size=4096, replace=False)]
    out = {
        "about": "FP64 oracle CG steady state of the 256^3 GRF tortuosity workload (written by make_golden.py)",
        "cg_relres": rel, "cg_iterations": iters, "seconds": time.time() - t0,
        "oracle_threads": oracle.num_threads(),
        "D_eff": d_eff, "tau": tau, "psi": psi, "J_in": red["J_in"], "J_out": red["J_out"],
        "n_active": red["n_active"],
        "samples_zyx": pick.tolist(),
        "samples_u": [float(u[z, y, x]) for z, y, x in pick],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grf256_steady.json")
    json.dump(out, open(path, "w"))
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("samples")}))


if __name__ == "__main__":
    main()
