"""Writes gap_sweep_oracle.json: the FP64 oracle's solutions of the benchmarked gap sweep.

Workload (Sec. 5.1, the sweep of Fig. sweep_im): two unit spheres at the 18 gaps
10^(-3 + 3 i / 17), N = 800 proxy Stokeslets on R_p = 0.63, M0 = 1600 basic nodes, images and
caps by the n_im rule (eq. image_est, <= 20 per contact), truncation 5e-12, and the three
relative motions squeeze / shear / counter-rotation.  Every problem is solved by the oracle's
matrix-free GMRES on eq. resistance (O3) to a relative residual of 1e-9, three orders below
the solve tolerance whose accuracy the stored values judge.

Stored per geometry: a fixed subset of the 500-point check grid on each sphere (every
`STRIDE`-th point).  Stored per problem: the forces and torques (Sec. 2.3 remark) and the
disturbance velocity u = G lambda at those check points (eq. lin_comb).

Only the oracle and the seeded input generators are called:
    python tests/golden/make_gap_sweep_oracle.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import geometry, solve  # noqa: E402
from paper_2407_03343_gb300 import workloads  # noqa: E402

PARAMS = dict(n_proxy=800, r_proxy=0.63, m_basic=1600)
MOTIONS = ("squeeze", "shear", "rotate")
TOL = 1e-9
STRIDE = 10
OUT = os.path.join(HERE, "gap_sweep_oracle.json")


def main():
    gaps = workloads.gap_sweep_gaps()
    out = {"params": PARAMS, "tol": TOL, "stride": STRIDE, "motions": list(MOTIONS), "gaps": gaps, "geometries": []}
    for g in gaps:
        t0 = time.time()
        d = geometry.build(workloads.two_spheres(g), 1.0, geometry.Params(**PARAMS))
        op = solve.Operator(d)
        x = np.concatenate([c[::STRIDE] for c in d.check])
        geo = {"gap": g, "contacts": len(d.contacts), "check_points": np.round(x, 15).tolist(), "problems": []}
        for m in MOTIONS:
            v, w = workloads.motion(m)
            sol = solve.solve_o3(d, v, w, op=op, tol=TOL)
            F, T = solve.forces_torques(d, sol.lam)
            u = solve.velocity(d, sol.lam, x)
            geo["problems"].append({"motion": m, "iters": int(sol.iters), "rel_residual": float(sol.rel_residual),
                                    "F": F.tolist(), "T": T.tolist(), "u": u.tolist()})
        out["geometries"].append(geo)
        print(f"gap {g:.4g}: {time.time() - t0:.1f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
