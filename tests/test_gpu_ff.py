"""The float-float fine propagator (df_sweep_kernel: every value an
unevaluated sum of two FP32 numbers, about 48 significant bits, on the FP32
pipes) of the ATM_FP64_FF and ATM_FP32_REFINED_FF precisions, against the FP64
oracle.

Bars: one application of the fine propagator <= 8 u_ff (1 + 4a), u_ff =
2^-48 the float-float unit roundoff and a = f D / dx^2 the largest line
coefficient (f = 1/2 for a PR half-step, 1 for backward Euler): the PR
right-hand side (1 - 2a) w + a (w[-1] + w[+1]) cancels terms of size 4a |w|
and the line solve's condition number is 1 + 4a, so relative rounding is
amplified by about 1 + 4a (at least 1e-13; measured values are printed, e.g.
5e-14 at 256^2 Allen-Cahn where 1 + 4a = 14); coarse levels (FP64 kernels)
<= 1e-13; iterates after j cycles <= 1e-12 (the FP64 bar); refined solves
<= 1e-7 against the oracle's sequential solution (the bar of every
FP32-propagation form)."""
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


KINDS = {
    "ac_pr": dict(kind="ac", dt=1e-4, m=(4, 4), k=3),
    "heat2d_pr": dict(kind="heat2d", dt=2e-4, m=(4,), lx=1.0, ly=0.7),
    "ac_split_fine": dict(kind="ac", dt=1e-4, m=(4,), fine_prop=atm.PROP_SPLIT_BE),
    "ac_pr_substeps3": dict(kind="ac", dt=1e-4, m=(4,), react_sub=(3, 0)),
}


def ff_bar(kw):
    """8 u_ff (1 + 4a) for the fine step of kw (see the module docstring)."""
    f = 0.5 if kw.get("fine_prop", atm.PROP_PR_ADI) == atm.PROP_PR_ADI else 1.0
    dx = min(kw.get("lx", 1.0) / kw["nx"], kw.get("ly", 1.0) / kw["ny"])
    a = f * kw["dt"] / dx ** 2
    return max(1e-13, 8 * 2.0 ** -48 * (1 + 4 * a))


@pytest.mark.parametrize("n", [64, 128, 256, 512])
@pytest.mark.parametrize("kind", sorted(KINDS))
def test_ff_propagator_matches_oracle(torch, kind, n):
    kw = dict(KINDS[kind], nx=n, ny=n, nt=65)
    oc, gp, gs = pair(precision=atm.FP64_FF, **kw)
    s = atm.Solver(gp, gs)
    assert s.sweep_config(0)["kernel"] == "float-float", s.sweep_config(0)
    x = I.uniform_field((5, n, n), 21, -1.0, 1.0)
    for level in range(len(kw["m"]) + 1):
        want = oracle.apply_prop(oc, level, x)
        got = s.apply_propagator(level, dev(torch, x)).cpu().numpy()
        errs = [rel_l2(got[j], want[j]) for j in range(5)]
        print(f"{kind} n={n} level={level}: max rel err {max(errs):.2e}")
        assert max(errs) <= (ff_bar(kw) if level == 0 else 1e-13), (level, errs, ff_bar(kw))
    s.close()


def test_ff_special_values(torch):
    """Zero states stay exactly zero; NaN propagates (divergence is seen); a
    state scaled by 1e30 (through the FP64 conversion) and one scaled by 1e-20
    (integer conversion) are as accurate as O(1) values (heat: Phi is linear).
    Float-float keeps FP32's exponent range: below ~2^-78 the low parts'
    rounding errors underflow, so a state scaled by 1e-30 keeps only about
    FP32 relative precision, and O(1) values beside tiny ones are unaffected."""
    oc, gp, gs = pair(kind="heat2d", nx=64, ny=64, dt=2e-4, nt=65, m=(4,), k=2, precision=atm.FP64_FF)
    s = atm.Solver(gp, gs)
    x = I.uniform_field((1, 64, 64), 22, -1.0, 1.0)
    z = np.zeros((1, 64, 64))
    nan = x.copy()
    nan[0, 10, 20] = np.nan
    mixed = x.copy()
    mixed[0, ::3, ::5] *= 1e-30
    batch = np.concatenate([z, nan, 1e-20 * x, 1e30 * x, x, 1e-30 * x, mixed])
    got = s.apply_propagator(0, dev(torch, batch)).cpu().numpy()
    want = oracle.apply_prop(oc, 0, np.concatenate([x, mixed]))
    bar = ff_bar(dict(nx=64, ny=64, dt=2e-4, lx=1.0, ly=1.0))
    assert np.all(got[0] == 0)
    assert np.isnan(got[1]).any()
    assert rel_l2(got[2] / 1e-20, want[0]) <= bar
    assert rel_l2(got[3] / 1e30, want[0]) <= bar
    assert rel_l2(got[4], want[0]) <= bar
    assert rel_l2(got[5] / 1e-30, want[0]) <= 1e-6
    assert rel_l2(got[6], want[1]) <= bar
    s.close()


FF_SOLVES = {
    "ac_3lvl_ragged": dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=300, m=(4, 4), k=3, nu=1),
    "heat2d_2lvl": dict(kind="heat2d", nx=128, ny=128, dt=1e-3, nt=129, m=(8,), k=3, nu=1),
    "ac_256_f": dict(kind="ac", nx=256, ny=256, dt=1e-4, nt=257, m=(16,), k=4, nu=0),
}


@pytest.mark.parametrize("case", sorted(FF_SOLVES))
def test_ff_iterates_match_oracle(torch, case):
    kw = dict(FF_SOLVES[case])
    n = kw["nx"]
    oc, gp, gs = pair(precision=atm.FP64_FF, tol=0.0, **kw)
    u0 = I.uniform_field((n, n), 23)
    for cycles in (1, 3):
        gs.max_iter = cycles
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        s.solve()
        got = s.solution().cpu().numpy()
        hist = s.residual_history()
        s.close()
        want = np.zeros_like(got)
        want[0] = u0
        it, ohist = oracle.solve(oc, want, cycles, 0.0)
        print(f"{case} cycles={cycles}: rel err {rel_l2(got, want):.2e}")
        assert rel_l2(got, want) <= 1e-12, (cycles, rel_l2(got, want))
        np.testing.assert_allclose(hist, ohist, rtol=1e-9)


@pytest.mark.parametrize("cpo", [False, True])
def test_ff_refined_reaches_the_oracle_solution(torch, cpo):
    kw = dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=1025, m=(8, 4), k=4, nu=1, tol=1e-9, max_iter=60,
              precision=atm.FP32_REFINED_FF, cpoint_only=cpo)
    oc, gp, gs = pair(**kw)
    s = atm.Solver(gp, gs)
    assert s.sweep_config(-1)["kernel"] == "float-float"
    u0 = I.uniform_field((128, 128), 24)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve()
    assert r["converged"], r
    seq = oracle.sequential(oc, u0)
    m0 = kw["m"][0]
    got = np.stack([s.solution(t, 1).cpu().numpy()[0] for t in range(0, kw["nt"], m0)])
    err = rel_l2(got, seq[::m0])
    print(f"refined float-float cpo={cpo}: {r['iterations']} passes, error {err:.2e}")
    assert err <= 1e-7
    s.close()
