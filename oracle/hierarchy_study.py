"""Residual histories of the oracle's AT-MGRIT / MGRIT on a window of the
large Allen-Cahn time hierarchy (dt = 2.5e-5, eps = 0.02) -- TEST
INFRASTRUCTURE ONLY: a study of why that hierarchy does not converge, run on
the CPU with the FP64 oracle.

    python -m oracle.hierarchy_study [n] [nt] [case,case,...]

Defaults: n = 256, nt = 16385, every case below; prints each case's residual
after cycles 0..4 (the first F-relaxation, then after each V-cycle).
"""
from __future__ import annotations

import sys
import time

import numpy as np

CASES = {
    "at_k16_fcf_exact": dict(m=(32, 4, 4), k=16, nu=1, exact=True),
    "mgrit_fcf_exact": dict(m=(32, 4, 4), k=0, nu=1, exact=True),
    "at_k16_3lvl": dict(m=(32, 4), k=16, nu=1, exact=True),
    "at_k16_fcf_substeps": dict(m=(32, 4, 4), k=16, nu=1, exact=False),
    "at_k16_m16": dict(m=(16, 4, 4), k=16, nu=1, exact=True),
    "at_k16_m8": dict(m=(8, 4, 4), k=16, nu=1, exact=True),
}


def run(n=256, nt=16385, names=None, cycles=4):
    import atm_inputs as I
    import oracle
    out = {}
    for name in names or list(CASES):
        cs = CASES[name]
        L = len(cs["m"]) + 1
        c = oracle.make_cfg(oracle.ALLEN_CAHN, n, n, dt=2.5e-5, nt=nt, eps=0.02, m=cs["m"], k=cs["k"],
                            nu=cs["nu"], react_exact=[l > 0 and cs["exact"] for l in range(L)])
        u = np.zeros((nt, n, n))
        u[0] = I.uniform_field((n, n), 0)
        t = time.time()
        _, hist = oracle.solve(c, u, cycles, 0.0)
        out[name] = [float(h) for h in hist]
        print(name, "%.1fs" % (time.time() - t), " ".join("%.3e" % h for h in hist), flush=True)
        del u
    return out


if __name__ == "__main__":
    a = sys.argv[1:]
    run(int(a[0]) if a else 256, int(a[1]) if len(a) > 1 else 16385, a[2].split(",") if len(a) > 2 else None)
