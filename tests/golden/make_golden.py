"""Writes tests/golden/c1_optimum.json from the FP64 oracle only.

Workload "c1": n=200, p=50, Toeplitz rho=0.1, k=5 ones, SNR=5, lambda2=0.01,
M = 1.5 ||ridge on the true support||_inf, lambda0 chosen so that the optimum
has 5 nonzeros, solved to gap 1e-6.  For each instance seed the script scans
lambda0 = f * lambda0_scale on a geometric grid, keeps the grid points whose
oracle optimum has exactly 5 nonzeros and records the middle one, with the
oracle's optimal support and objective.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen  # noqa: E402
from oracle import bnb  # noqa: E402

GRID = [0.4, 0.3, 0.2, 0.15, 0.1, 0.07, 0.05, 0.035, 0.025]


def main(instances=(0, 1, 2)):
    out = []
    cfg = datagen.CONFIGS["c1"]
    for inst_id in instances:
        inst = datagen.config_instance("c1", inst_id)
        lam2 = cfg["lam2"]
        M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
        scale = datagen.lambda0_scale(inst.X, inst.y, lam2)
        hits = []
        for f in GRID:
            res = bnb.solve(inst.X, inst.y, f * scale, lam2, M, gap=1e-6)
            if np.count_nonzero(res.beta) == cfg["k"] and res.status == "optimal":
                hits.append((f, res))
        f, res = hits[len(hits) // 2]
        out.append(dict(instance=inst_id, seed=inst.seed, lambda0=f * scale, lambda2=lam2, M=M,
                        gap=1e-6, support=[int(i) for i in np.nonzero(res.beta)[0]],
                        objective=res.ub, lower_bound=res.lb, oracle_nodes=res.nodes))
    with open(os.path.join(HERE, "c1_optimum.json"), "w") as fh:
        json.dump(dict(workload="c1", source="oracle.bnb (FP64)", cases=out), fh, indent=1)


if __name__ == "__main__":
    main()
