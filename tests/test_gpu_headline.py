"""The 256^2 Allen-Cahn workload at its full size (4097 points, m = (16, 16),
k = 8, FCF, three levels) against the FP64 oracle, in the configurations the
benchmark times.

* The benchmark's own path -- FP32 propagation inside the FP64 refinement
  loop, C-point storage, five inner cycles, autotuned level-0 kernel -- solved
  to ||r||_2 <= 1e-8: its C-points (all 257) and its final state against the
  oracle's sequential solution (the fixed point of Sec. 2) at relative L2
  <= 1e-7, state by state.
* The FP64 solver: every point of the level-0 iterate after one and two
  cycles against the oracle's literal Algorithm 2 at <= 1e-12.
* Every building block of one cycle (Algorithm 2) at full size: level-0
  F/C/F-relaxation, restriction to level 1 (v, r, g), the level-1 relaxations
  and restriction to level 2, the 17 local chains of the coarsest level (k = 8)
  and the correction, each against the oracle's stage at <= 1e-12."""
import numpy as np
import pytest

import atm_inputs as I
import bench
import oracle
import paper_2107_09596_gb300 as atm
from helpers import pair, rel_l2

pytestmark = pytest.mark.gpu

W = bench.WORKLOADS["allen_cahn_256"]
NT, N, M0 = W["nt"], W["n"], W["m"][0]


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    atm._build.build()
    atm.load()
    return torch


@pytest.fixture(scope="module")
def sequential():
    """The oracle's sequential solution of the workload (seed 0), C-points only."""
    oc, _, _ = pair(kind="ac", nx=N, ny=N, dt=W["dt"], nt=NT, eps=W["eps"], m=W["m"], k=W["k"], nu=W["nu"])
    u = oracle.sequential(oc, I.uniform_field((N, N), 0))
    return u[::M0].copy()


@pytest.mark.parametrize("prec, sweep", [("fp32r", "auto"), ("fp32r", "persistent"), ("fp32rf", "auto")])
def test_bench_path_matches_the_oracle_sequential_solution(torch, sequential, prec, sweep):
    prob, desc = bench.make_desc(atm, W, "at", bench.PRECISIONS[prec](atm), profile=True, cpoint=True,
                                 sweep=sweep)
    s = atm.Solver(prob, desc)
    s.set_initial_condition(torch.as_tensor(bench.initial_condition(W, 0), device="cuda:0"))
    res = s.solve()
    assert res["converged"] and res["final_residual"] <= W["tol"], res
    assert s.sweep_config(0)["kernel"] in ("fused", "split", "persistent")
    got = np.stack([s.solution(t, 1).cpu().numpy()[0] for t in range(0, NT, M0)])
    assert got.shape == sequential.shape
    errs = [rel_l2(got[i], sequential[i]) for i in range(got.shape[0])]
    assert max(errs) <= 1e-7, (int(np.argmax(errs)) * M0, max(errs))
    assert rel_l2(got, sequential) <= 1e-7
    # the final state is the last C-point (4096 = 256 * 16)
    assert rel_l2(s.solution(NT - 1, 1).cpu().numpy()[0], sequential[-1]) <= 1e-7
    s.close()


def test_fp64_iterates_at_full_size(torch):
    oc, gp, gs = pair(kind="ac", nx=N, ny=N, dt=W["dt"], nt=NT, eps=W["eps"], m=W["m"], k=W["k"], nu=W["nu"],
                      tol=0.0, max_iter=2)
    u0 = I.uniform_field((N, N), 0)
    u = np.zeros((NT, N, N))
    u[0] = u0
    for cycles in (1, 2):
        gs.max_iter = cycles
        s = atm.Solver(gp, gs)
        s.set_initial_condition(torch.as_tensor(u0, device="cuda:0"))
        s.solve()
        got = s.solution().cpu().numpy()
        s.close()
        ou = u.copy()
        oracle.solve(oc, ou, cycles, 0.0)
        assert rel_l2(got, ou) <= 1e-12, (cycles, rel_l2(got, ou))
        assert rel_l2(got[::M0], ou[::M0]) <= 1e-12
        del got, ou


def test_every_stage_at_full_size(torch):
    oc, gp, gs = pair(kind="ac", nx=N, ny=N, dt=W["dt"], nt=NT, eps=W["eps"], m=W["m"], k=W["k"], nu=W["nu"])
    s = atm.Solver(gp, gs)
    u = np.zeros((NT, N, N))
    u[0] = I.uniform_field((N, N), 0)
    u[M0::M0] = I.uniform_field((NT // M0, N, N), 9, -0.5, 0.5)   # a C-point guess
    s.level_write(0, atm.ARRAY_U, torch.as_tensor(u, device="cuda:0"))
    tol = 1e-12

    def chk(level, array, want):
        got = s.level_read(level, array).cpu().numpy()
        assert got.shape == want.shape
        assert rel_l2(got, want) <= tol, (level, array, rel_l2(got, want))

    s.run_stage(atm.STAGE_F_RELAX, 0)
    oracle.frelax_level(oc, 0, u)
    s.run_stage(atm.STAGE_C_RELAX, 0)
    oracle.crelax_level(oc, 0, u)
    s.run_stage(atm.STAGE_F_RELAX, 0)
    oracle.frelax_level(oc, 0, u)
    chk(0, atm.ARRAY_U, u)
    s.run_stage(atm.STAGE_RESTRICT, 0)
    v1, r1, g1 = oracle.restrict_level(oc, 0, u)
    for a, want in ((atm.ARRAY_V, v1), (atm.ARRAY_R, r1), (atm.ARRAY_G, g1)):
        chk(1, a, want)
    u1 = v1.copy()
    s.run_stage(atm.STAGE_F_RELAX, 1)
    oracle.frelax_level(oc, 1, u1, g1)
    s.run_stage(atm.STAGE_C_RELAX, 1)
    oracle.crelax_level(oc, 1, u1, g1)
    s.run_stage(atm.STAGE_F_RELAX, 1)
    oracle.frelax_level(oc, 1, u1, g1)
    chk(1, atm.ARRAY_U, u1)
    s.run_stage(atm.STAGE_RESTRICT, 1)
    v2, r2, g2 = oracle.restrict_level(oc, 1, u1, g1)
    for a, want in ((atm.ARRAY_V, v2), (atm.ARRAY_R, r2), (atm.ARRAY_G, g2)):
        chk(2, a, want)
    assert v2.shape[0] == 17
    s.run_stage(atm.STAGE_COARSEST)
    u2 = oracle.coarsest_level(oc, 2, v2, r2, g2)
    chk(2, atm.ARRAY_U, u2)
    s.run_stage(atm.STAGE_CORRECT, 1)
    u1[::M0] = u1[::M0] + (u2 - v2)
    chk(1, atm.ARRAY_U, u1)
    s.run_stage(atm.STAGE_F_RELAX, 1)
    oracle.frelax_level(oc, 1, u1, g1)
    chk(1, atm.ARRAY_U, u1)
    s.run_stage(atm.STAGE_CORRECT, 0)
    u[::M0] = u[::M0] + (u1 - v1)
    s.run_stage(atm.STAGE_F_RELAX, 0)
    oracle.frelax_level(oc, 0, u)
    chk(0, atm.ARRAY_U, u)
    s.close()
