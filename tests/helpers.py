"""Test glue: build matching oracle and GPU descriptions of one problem."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2107_09596_gb300 as atm

KIND = {"heat1d": (oracle.HEAT1D, atm.HEAT1D), "heat2d": (oracle.HEAT2D, atm.HEAT2D),
        "ac": (oracle.ALLEN_CAHN, atm.ALLEN_CAHN)}


def pair(kind="heat1d", nx=127, ny=1, lx=1.0, ly=1.0, dt=1.0 / 1024, nt=1025, eps=0.02,
         m=(8,), k=4, nu=1, algorithm="at", fine_prop=atm.PROP_PR_ADI,
         coarse_prop=atm.PROP_SPLIT_BE, react_sub=None, coarse_reaction=atm.REACT_EXACT,
         precision=atm.FP64, tol=0.0, max_iter=10, use_graph=True, cpoint_only=False,
         sweep_kernel=atm.SWEEP_AUTO):
    ok, gk = KIND[kind]
    L = len(m) + 1
    prop = [fine_prop if l == 0 else coarse_prop for l in range(L)]
    ok_k = k if algorithm == "at" else 0
    exact = [l > 0 and coarse_reaction == atm.REACT_EXACT for l in range(L)]
    oc = oracle.make_cfg(ok, nx, ny, lx=lx, ly=ly, dt=dt, nt=nt, eps=eps, m=m, k=ok_k, nu=nu,
                         prop=prop, react_sub=react_sub, react_exact=exact)
    gp = atm.make_problem(gk, nx, ny if kind != "heat1d" else 1, lx=lx, ly=ly, dt=dt,
                          nt_points=nt, eps=eps)
    alg = {"at": atm.AT_MGRIT, "mgrit": atm.MGRIT, "seq": atm.SEQUENTIAL}[algorithm]
    gs = atm.make_solver(alg, m=m, k=k, nu=nu, fine_prop=fine_prop, coarse_prop=coarse_prop,
                         reaction_substeps=react_sub, coarse_reaction=coarse_reaction,
                         tol=tol, max_iter=max_iter,
                         precision=precision, use_graph=use_graph, cpoint_only=cpoint_only,
                         sweep_kernel=sweep_kernel)
    return oc, gp, gs


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
