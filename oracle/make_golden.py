"""Write the oracle's residual histories for the benchmark workloads to
tests/golden/oracle_histories.json.  Calls only the oracle (FP64 CPU) and the
seeded input generators; run from the repository root:

    python -m oracle.make_golden [--skip-cfg2]

Workloads (seeded, synthetic):
  cfg1: 1D heat, nx=127 interior points on [0,1], Dirichlet, backward Euler,
        1025 points, dt=1/1024, two levels, m=8, FCF, k=4 (and k=5, MGRIT),
        u0 = sin(pi x) + 0.1 * 8 seeded sine modes, zero initial guess.
  cfg2: 2D Allen-Cahn, 256^2 periodic [0,1)^2, eps=0.02, PR-ADI fine step with
        explicit reaction, split-BE ADI coarse steps after the exact reaction flow,
        4097 points, dt=1e-4, three levels m=(16,16), FCF, k=8 (and MGRIT),
        u0 ~ U(-0.05, 0.05) seed 0, zero initial guess, tol 1e-8.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import atm_inputs as I  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "oracle_histories.json")


def run(cfg, u0, max_iter, tol):
    u = np.zeros((cfg.nt,) + oracle.state_shape(cfg))
    u[0] = u0
    t = time.time()
    it, hist = oracle.solve(cfg, u, max_iter, tol)
    return {"iterations": int(it), "history": [float(h) for h in hist],
            "seconds": round(time.time() - t, 2), "threads": oracle.num_threads()}


def main():
    out = {"generator": "oracle/make_golden.py"}
    u0 = I.heat1d_initial_condition(127, 0)
    for name, k in (("cfg1_at_k4", 4), ("cfg1_at_k5", 5), ("cfg1_mgrit", 0)):
        c = oracle.make_cfg(oracle.HEAT1D, 127, dt=1 / 1024, nt=1025, m=(8,), k=k, nu=1)
        out[name] = run(c, u0, 60, 1e-10)
        print(name, out[name]["iterations"], flush=True)
    if "--skip-cfg2" not in sys.argv:
        u0 = I.uniform_field((256, 256), 0)
        for name, k in (("cfg2_at_k8", 8), ("cfg2_mgrit", 0)):
            c = oracle.make_cfg(oracle.ALLEN_CAHN, 256, 256, dt=1e-4, nt=4097, eps=0.02,
                                m=(16, 16), k=k, nu=1, react_exact=[0, 1, 1])
            out[name] = run(c, u0, 40, 1e-8)
            print(name, out[name]["iterations"], out[name]["seconds"], flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
