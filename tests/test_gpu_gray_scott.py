"""Gray-Scott (Sec. 5.1) on the GPU against the oracle: the backward Euler
Newton propagator on every level, the per-iteration iterates and residual
histories of AT-MGRIT / MGRIT cycles, nested iteration, C-point storage and
the device-side loop.

Both sides solve each step's nonlinear system to ||G||_2 <= 1e-12 (absolute),
the oracle by Newton with exact sparse solves, the GPU by Newton with GMRES;
the step results then agree to about that tolerance times ||M^-1|| (<= a few),
and a space-time iterate accumulates at most one such error per step, hence
the relative L2 bound 1e-10 below."""
import numpy as np
import pytest

import atm_inputs as I
import oracle
import paper_2107_09596_gb300 as atm
from helpers import rel_l2

pytestmark = pytest.mark.gpu

PAR = dict(du=8e-5, dv=4e-5, feed=0.024, kill=0.06)
DT = 256.0 / 16383.0
NEWTON_TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    atm._build.build()
    atm.load()
    return torch


def dev(torch, x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def gs_pair(nx=32, ny=32, lx=2.5, ly=2.5, dt=DT, nt=129, m=(8,), k=4, nu=1, algorithm="at",
            tol=0.0, max_iter=5, use_graph=True, cpoint_only=False, nested=False, newton_tol=NEWTON_TOL):
    oc = oracle.make_cfg(oracle.GRAY_SCOTT, nx, ny, lx=lx, ly=ly, dt=dt, nt=nt, m=m,
                         k=(k if algorithm == "at" else 0), nu=nu,
                         gs=dict(PAR, tol=newton_tol, max_iter=50))
    gp = atm.make_problem(atm.GRAY_SCOTT, nx, ny, lx=lx, ly=ly, dt=dt, nt_points=nt,
                          newton_tol=newton_tol, newton_max_iter=50, **PAR)
    alg = {"at": atm.AT_MGRIT, "mgrit": atm.MGRIT, "seq": atm.SEQUENTIAL}[algorithm]
    gs = atm.make_solver(alg, m=m, k=k, nu=nu, tol=tol, max_iter=max_iter, use_graph=use_graph,
                         cpoint_only=cpoint_only, nested=nested)
    return oc, gp, gs


def initial_state(nx, ny):
    return I.gray_scott_initial_condition(nx, ny)


@pytest.mark.parametrize("shape", [(32, 32), (40, 24), (128, 128)])
def test_propagator_matches_oracle_on_every_level(torch, shape):
    nx, ny = shape
    lx, ly = 2.5, 2.5 * ny / nx
    m = (8, 8)
    oc, gp, gs = gs_pair(nx=nx, ny=ny, lx=lx, ly=ly, nt=129, m=m, k=2)
    s = atm.Solver(gp, gs)
    assert s.sweep_config(0)["kernel"] == "newton"
    states = [initial_state(nx, ny)] + [I.gray_scott_random_state(nx, ny, seed) for seed in (11, 12)]
    x = np.stack(states)
    for level in range(3):
        got = s.apply_propagator(level, dev(torch, x)).cpu().numpy()
        want = oracle.apply_prop(oc, level, x)
        err = np.abs(got - want).max()
        print(f"\n{nx}x{ny} level {level} (D = {oracle.level_dt(oc, level):.4g}): max |GPU - oracle| = {err:.2e}")
        assert err <= 1e-10, (level, err)
    st = s.newton_stats()
    assert st["steps"] == 3 * len(states) and st["failures"] == 0
    assert st["newton"] >= st["steps"] and st["gmres"] >= st["newton"]


SOLVE_CASES = {
    "at_2lvl_fcf": dict(nt=129, m=(8,), k=4, nu=1),
    "at_3lvl_f_ragged": dict(nt=150, m=(4, 4), k=3, nu=0),
    "mgrit_2lvl_fcf": dict(nt=129, m=(8,), k=4, nu=1, algorithm="mgrit"),
}


@pytest.mark.parametrize("case", sorted(SOLVE_CASES))
def test_solve_iterates_match_oracle(torch, case):
    kw = SOLVE_CASES[case]
    nt = kw["nt"]
    u0 = initial_state(32, 32)
    for j in (1, 3):
        oc, gp, gs = gs_pair(max_iter=j, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        r = s.solve()
        assert r["iterations"] == j
        got = s.solution().cpu().numpy()
        want = np.zeros((nt, 2, 32, 32))
        want[0] = u0
        it, hist = oracle.solve(oc, want, j, 0.0)
        err = rel_l2(got, want)
        print(f"\n{case} after {j}: rel L2 {err:.2e}, residuals {s.residual_history()} / {hist}")
        assert err <= 1e-10, (j, err)
        np.testing.assert_allclose(s.residual_history(), hist, rtol=1e-6, atol=1e-10)


def test_converged_solution_is_sequential(torch):
    oc, gp, gs = gs_pair(nt=129, m=(8,), k=4, nu=1, tol=1e-9, max_iter=30)
    u0 = initial_state(32, 32)
    s = atm.Solver(gp, gs)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve(allow_not_converged=False)
    seq = oracle.sequential(oc, u0)
    got = s.solution().cpu().numpy()
    print(f"\nconverged in {r['iterations']} cycles; rel L2 to sequential {rel_l2(got, seq):.2e}")
    assert rel_l2(got, seq) <= 1e-9
    # sequential stepping on the GPU
    _, gp2, gs2 = gs_pair(nt=129, algorithm="seq")
    q = atm.Solver(gp2, gs2)
    q.set_initial_condition(dev(torch, u0))
    q.solve()
    assert rel_l2(q.solution().cpu().numpy(), seq) <= 1e-10


@pytest.mark.parametrize("graph", [1, 2])
def test_nested_iteration_with_cpoint_storage(torch, graph):
    """The paper's Gray-Scott runs start from nested iteration; with C-point
    storage and the device-side loop the C-points match the oracle's nested
    guess followed by the same cycles."""
    kw = dict(nt=129, m=(4, 4), k=3, nu=1)
    u0 = initial_state(32, 32)
    for cycles in (1, 2):
        oc, gp, gs = gs_pair(max_iter=cycles, use_graph=graph, cpoint_only=True, nested=True, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        s.solve()
        want = np.zeros((kw["nt"], 2, 32, 32))
        want[0] = u0
        oracle.nested_guess(oc, want)
        _, hist = oracle.solve(oc, want, cycles, 0.0)
        cp = np.arange(0, kw["nt"], 4)
        got = s.solution().cpu().numpy()
        err = rel_l2(got[cp], want[cp])
        print(f"\nnested + {cycles} cycles (graph {graph}): rel L2 at C-points {err:.2e}")
        assert err <= 1e-10
        np.testing.assert_allclose(s.residual_history(), hist, rtol=1e-6, atol=1e-10)


def test_invalid_gray_scott_options_are_rejected(torch):
    _, gp, gs = gs_pair()
    gs.precision = atm.FP32
    with pytest.raises(atm.AtmError):
        atm.Solver(gp, gs)
    _, gp, gs = gs_pair()
    gs.sweep_kernel = atm.SWEEP_FUSED
    with pytest.raises(atm.AtmError):
        atm.Solver(gp, gs)
    _, gp, gs = gs_pair(nx=4)
    with pytest.raises(atm.AtmError):
        atm.Solver(gp, gs)


def test_paper_iteration_counts_at_full_size(torch):
    """Sec. 5.1 at the paper's size (128^2, 16384 points, nested iteration,
    Newton tolerance 1e-10, space-time residual 1e-7): the iteration counts
    printed in Tables 1 and 2."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    u0 = initial_state(128, 128)
    for case in gold["gray_scott_iterations"]["cases"]:
        _, gp, gs = gs_pair(nx=128, ny=128, nt=16384, m=tuple(case["m"]), k=max(case["k"], 1),
                            nu=case["nu"], algorithm=case["algorithm"], tol=1e-7, max_iter=30,
                            use_graph=2, cpoint_only=True, nested=True, newton_tol=1e-10)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        r = s.solve()
        print(f"\n{case['name']}: {r['iterations']} cycles (paper {case['iterations']}), "
              f"residual {r['final_residual']:.2e}")
        assert r["converged"] and r["iterations"] == case["iterations"]
        assert s.newton_stats()["failures"] == 0
        s.close()
