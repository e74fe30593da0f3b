"""Writes tests/golden/reactive512_2000.json with the FP64 oracle only.

The 512^3 two-species reactive workload (Boolean polydisperse spheres at pore
fraction 0.40; A diffuses with D = 1 and reacts A -> B at the surface with
k = 0.05 times the smoothed delta weight; B diffuses with D = 0.5 and decays
at 0.001; A = 1 for x < 32, B = 0; closed box; dt = 0.9 x the explicit
limit) is advanced 2000 forward-Euler steps by the dense FP64 oracle, the
steps Sec. 3.5's surface-sink model is run for in the workload.  The script
stores, per species, the mass, the maximum, the sum over every x plane (the
profile along the transport direction) and the values at seeded sample
voxels: 4096 over all active voxels, 2048 in the front region 16 <= x < 96
where A and B change fastest, and 2048 on surface-band voxels (0 < phi < 1,
where the reaction acts).  The oracle threads and the wall time are stored
as well.  Run: python tests/golden/make_golden_reactive512.py [steps]
(takes tens of minutes on a few cores and about 5 GB of host memory).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import reactive512  # noqa: E402


def main():
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 2000
    t0 = time.time()
    phi, u0, phys = reactive512()
    P = oracle.Problem(phi, phys)
    u = P.run(u0, steps)
    secs = time.time() - t0
    red = P.reduce(u)
    act = P.active > 0
    rng = np.random.default_rng(5151)
    idx_all = np.argwhere(act)
    pick_all = idx_all[rng.choice(len(idx_all), size=4096, replace=False)]
    front = act.copy()
    front[:, :, :16] = False
    front[:, :, 96:] = False
    idx_front = np.argwhere(front)
    pick_front = idx_front[rng.choice(len(idx_front), size=2048, replace=False)]
    band = act & (P.w > 0)
    idx_band = np.argwhere(band)
    pick_band = idx_band[rng.choice(len(idx_band), size=2048, replace=False)]
    pick = np.concatenate([pick_all, pick_front, pick_band])
    out = {
        "about": ("FP64 oracle state of the 512^3 two-species reactive workload after %d steps "
                  "(written by make_golden_reactive512.py)" % steps),
        "steps": steps, "dt": phys.dt, "seconds": secs, "oracle_threads": oracle.num_threads(),
        "n_active": int(act.sum()),
        "mass": [float(r["mass"]) for r in red],
        "max": [float(u[s].max()) for s in range(2)],
        "x_profile": [u[s].sum(axis=(0, 1)).tolist() for s in range(2)],
        "samples_zyx": pick.tolist(),
        "samples_kind": ["all"] * len(pick_all) + ["front"] * len(pick_front) + ["band"] * len(pick_band),
        "samples_u": [[float(u[s][z, y, x]) for z, y, x in pick] for s in range(2)],
    }
    name = "reactive512_%d.json" % steps
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    json.dump(out, open(path, "w"))
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("samples") and k != "x_profile"}))


if __name__ == "__main__":
    main()
