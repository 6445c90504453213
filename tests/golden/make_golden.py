"""Writes tests/golden/poisson_small_oracle.json: sampled values of the
oracle's solution of the 32^3 uniform Neumann workload.  It calls only the
oracle (and the seeded input generator); the stored values pin the oracle
against unintended change, never against the CUDA path.

    python tests/golden/make_golden.py
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2502_06296_gb300 import synth  # noqa: E402


def main():
    cfg = synth.SMALL
    f = synth.small_rhs(cfg)
    dz = synth.grid_dz(cfg)
    p = oracle.poisson_solve(f, cfg["lx"], cfg["ly"], dz, oracle.NEUMANN)
    idx = [(0, 0, 0), (31, 31, 31), (5, 17, 29), (16, 0, 8), (30, 2, 1), (11, 22, 3)]
    out = {"workload": cfg["name"], "seed": cfg["seed"], "bc": "neumann",
           "source": "oracle.poisson_solve on synth.small_rhs(synth.SMALL)",
           "samples": [{"zyx": list(i), "p": float(p[i])} for i in idx],
           "max_abs_p": float(np.max(np.abs(p))), "sum_p": float(p.sum())}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson_small_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
