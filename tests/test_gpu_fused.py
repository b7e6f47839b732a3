"""The fused whole-propagator kernel (one thread-block cluster per state, the
state held in shared memory) against the FP64 oracle and against the split
row/column kernels.  Both FP32 paths perform the same operations; they differ
in how the column recurrences are chunked, hence in FP32 rounding only:
relative L2 <= 3e-6 per application against the oracle (the FP32 bar of the
split kernels), and solves reach the same fixed point."""
import numpy as np
import pytest

import atm_inputs as I
import oracle
import paper_2107_09596_gb300 as atm
from helpers import pair, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    atm._build.build()
    atm.load()
    return torch


def dev(torch, x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


GRIDS = [64, 128, 256, 512]
KINDS = {
    "ac_pr_exact": dict(kind="ac", dt=1e-4, m=(4, 4), k=3),
    "ac_pr_substeps": dict(kind="ac", dt=1e-4, m=(4, 4), k=3, coarse_reaction=atm.REACT_SUBSTEPS),
    "heat2d_pr": dict(kind="heat2d", dt=2e-4, m=(4,), lx=1.0, ly=0.7),
    "ac_split_fine": dict(kind="ac", dt=1e-4, m=(4,), fine_prop=atm.PROP_SPLIT_BE),
}


def fp32_tol(kw, level):
    """FP32 bar of one application: the line solves amplify relative rounding
    by their condition number 1 + 4a (a = f D / dx^2 with f = 1/2 for a PR
    half-step, 1 for backward Euler); 2.5e-7 (1 + 4a), at least 3e-6 (the bar
    of the split kernels at 256^2, where 1 + 4a ~ 14 on level 0)."""
    D = kw["dt"]
    for j in range(level):
        D *= kw["m"][j]
    pr = level == 0 and kw.get("fine_prop", atm.PROP_PR_ADI) == atm.PROP_PR_ADI
    dx = min(kw.get("lx", 1.0) / kw["nx"], kw.get("ly", 1.0) / kw["ny"])
    a = (0.5 if pr else 1.0) * D / dx ** 2
    return max(3e-6, 2.5e-7 * (1 + 4 * a))


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("kind", sorted(KINDS))
def test_fused_propagator_matches_oracle_and_split(torch, kind, n):
    kw = dict(KINDS[kind], nx=n, ny=n, nt=65)
    oc, gp, gf = pair(precision=atm.FP32, sweep_kernel=atm.SWEEP_FUSED, **kw)
    _, _, gsp = pair(precision=atm.FP32, sweep_kernel=atm.SWEEP_SPLIT, **kw)
    f, sp = atm.Solver(gp, gf), atm.Solver(gp, gsp)
    x = I.uniform_field((3, n, n), 11, -1.0, 1.0)
    for level in range(len(kw["m"]) + 1):
        tol = fp32_tol(kw, level)
        want = oracle.apply_prop(oc, level, x)
        got = f.apply_propagator(level, dev(torch, x)).cpu().numpy()
        ref = sp.apply_propagator(level, dev(torch, x)).cpu().numpy()
        for j in range(3):
            ef, es = rel_l2(got[j], want[j]), rel_l2(ref[j], want[j])
            print(f"{kind} n={n} level={level} fused {ef:.2e} split {es:.2e} tol {tol:.1e}")
            assert ef <= tol and es <= tol, (level, j, ef, es, tol)
            # and the fused kernel is as accurate as the split kernels
            assert ef <= 2 * es + 1e-6, (level, j, ef, es)


@pytest.mark.parametrize("n", [64, 128, 256])
def test_fused_fp32_solve_reaches_the_fp32_fixed_point(torch, n):
    # FP32 residual floor ~ eps_32 |u| sqrt(#C-point values): stop well above it
    kw = dict(kind="ac", nx=n, ny=n, dt=1e-4, nt=129, m=(4, 4), k=4, nu=1, tol=1e-4 * n / 64, max_iter=40,
              precision=atm.FP32)
    u0 = I.uniform_field((n, n), 12)
    res = {}
    for sk in (atm.SWEEP_FUSED, atm.SWEEP_SPLIT):
        oc, gp, gs = pair(sweep_kernel=sk, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        r = s.solve()
        print(f"n={n} sweep_kernel={sk}: {r['iterations']} cycles, residual {r['final_residual']:.3e}")
        assert r["converged"], (sk, r)
        res[sk] = (r, s.solution().cpu().numpy())
    seq = oracle.sequential(oc, u0)
    for sk, (r, u) in res.items():
        assert rel_l2(u, seq) <= 1e-4, (sk, rel_l2(u, seq))
    assert abs(res[atm.SWEEP_FUSED][0]["iterations"] - res[atm.SWEEP_SPLIT][0]["iterations"]) <= 1


@pytest.mark.parametrize("cpo", [False, True])
def test_fused_inner_cycle_of_the_refined_mode(torch, cpo):
    """The refined mode's FP32 inner cycle on fused kernels (increments around
    a base; with C-point storage the base chain is regenerated in launches of
    its own) still reaches the FP64 fixed point within 1e-7."""
    kw = dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9, max_iter=60,
              precision=atm.FP32_REFINED, sweep_kernel=atm.SWEEP_FUSED, cpoint_only=cpo)
    oc, gp, gs = pair(**kw)
    s = atm.Solver(gp, gs)
    u0 = I.uniform_field((128, 128), 13)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve()
    assert r["converged"], r
    seq = oracle.sequential(oc, u0)
    assert rel_l2(s.solution().cpu().numpy(), seq) <= 1e-7


def test_fused_residual_norm_matches_split(torch):
    """The fused kernel's per-CTA residual sums give the same norm as the split
    kernels' (same residual values up to FP32 rounding)."""
    kw = dict(kind="ac", nx=256, ny=256, dt=1e-4, nt=257, m=(16, 4), k=4, nu=1, tol=0.0, max_iter=3,
              precision=atm.FP32)
    u0 = I.uniform_field((256, 256), 14)
    hs = []
    for sk in (atm.SWEEP_FUSED, atm.SWEEP_SPLIT):
        _, gp, gs = pair(sweep_kernel=sk, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        s.solve()
        hs.append(s.residual_history())
    np.testing.assert_allclose(hs[0], hs[1], rtol=1e-3)


@pytest.mark.parametrize("inner", [2, 3])
def test_refined_with_several_inner_cycles(torch, inner):
    """Several FP32 V-cycles on the correction per FP64 residual: the same FP64
    fixed point (<= 1e-7 against the oracle) with fewer FP64 residual passes."""
    kw = dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9, max_iter=60,
              precision=atm.FP32_REFINED)
    u0 = I.uniform_field((64, 64), 15)
    res = {}
    for ic in (1, inner):
        oc, gp, gs = pair(**kw)
        gs.refine_inner_cycles = ic
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        r = s.solve()
        assert r["converged"], (ic, r)
        res[ic] = (r, s.solution().cpu().numpy())
    seq = oracle.sequential(oc, u0)
    assert rel_l2(res[inner][1], seq) <= 1e-7
    assert res[inner][0]["iterations"] < res[1][0]["iterations"], (res[1][0], res[inner][0])


@pytest.mark.parametrize("relax", [0, 1])
def test_refined_inner_coarse_relaxation(torch, relax):
    """The coarse levels of the FP32 inner cycles relaxed by F (refine_coarse_relax
    = 0, the default) or, like level 0, by FCF (1): the same FP64 fixed point
    (<= 1e-7 against the oracle's sequential solution)."""
    kw = dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=257, m=(8, 4), k=4, nu=1, tol=1e-9, max_iter=60,
              precision=atm.FP32_REFINED_FF, cpoint_only=True)
    oc, gp, gs = pair(**kw)
    gs.refine_coarse_relax = relax
    s = atm.Solver(gp, gs)
    u0 = I.uniform_field((128, 128), 16)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve()
    assert r["converged"], r
    seq = oracle.sequential(oc, u0)
    assert rel_l2(s.solution().cpu().numpy(), seq) <= 1e-7


CHAIN_CASES = {
    "ac64_ragged_full": dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=300, m=(4, 4), k=3, nu=1),
    "ac128_cpoint": dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=257, m=(8, 4), k=4, nu=1, cpoint_only=True),
    "heat256_f": dict(kind="heat2d", nx=256, ny=256, dt=2e-4, nt=257, m=(16,), k=4, nu=0),
    "ac256_3lvl": dict(kind="ac", nx=256, ny=256, dt=1e-4, nt=513, m=(16, 4), k=4, nu=1),
}


@pytest.mark.parametrize("case", sorted(CHAIN_CASES))
def test_chain_kernel_solves_like_the_fused_kernel(torch, case):
    """F-relaxations as chains (one launch; each interval's steps on its state
    in shared memory) reach the same FP32 fixed point as step-by-step fused
    launches and the FP64 sequential solution within the FP32 bar."""
    kw = dict(CHAIN_CASES[case], precision=atm.FP32, tol=0.0, max_iter=6)
    n = kw["nx"]
    u0 = I.uniform_field((n, n), 31)
    sols = {}
    for sk in (atm.SWEEP_CHAIN, atm.SWEEP_FUSED):
        oc, gp, gs = pair(sweep_kernel=sk, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        s.solve()
        sols[sk] = (s.solution().cpu().numpy(), s.residual_history())
    assert rel_l2(sols[atm.SWEEP_CHAIN][0], sols[atm.SWEEP_FUSED][0]) <= 1e-5
    np.testing.assert_allclose(sols[atm.SWEEP_CHAIN][1], sols[atm.SWEEP_FUSED][1], rtol=1e-3)
    # after 6 cycles both sit at the same iterate; the FP64 oracle after 6 cycles agrees to FP32
    want = np.zeros_like(sols[atm.SWEEP_CHAIN][0])
    want[0] = u0
    oracle.solve(oc, want, 6, 0.0)
    assert rel_l2(sols[atm.SWEEP_CHAIN][0], want) <= 1e-4


def test_chain_kernel_in_the_refined_inner_cycles(torch):
    kw = dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9, max_iter=40,
              precision=atm.FP32_REFINED, sweep_kernel=atm.SWEEP_CHAIN, cpoint_only=True)
    oc, gp, gs = pair(**kw)
    s = atm.Solver(gp, gs)
    u0 = I.uniform_field((128, 128), 32)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve()
    assert r["converged"], r
    assert rel_l2(s.solution().cpu().numpy(), oracle.sequential(oc, u0)) <= 1e-7
