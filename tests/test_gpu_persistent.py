"""The persistent cluster kernel (fused_persist_kernel: as many clusters as
fit on the GPU walk the states of a launch; the next state's input arrives in
a second shared-memory tile while the current one is solved) against the FP64
oracle and the split kernels.  Launches carry more states than the grid has
clusters, so that every cluster solves several states in a row (the
double-buffered path).  FP32 bars as for the fused kernel (test_gpu_fused)."""
import numpy as np
import pytest

import atm_inputs as I
import oracle
import paper_2107_09596_gb300 as atm
from helpers import pair, rel_l2
from test_gpu_fused import KINDS, fp32_tol

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


# states per launch: more than the persistent grid's clusters at every size
NSTATES = {64: 700, 128: 400, 256: 200, 512: 24}


@pytest.mark.parametrize("n", [64, 128, 256, 512])
@pytest.mark.parametrize("kind", sorted(KINDS))
def test_persistent_propagator_matches_oracle_and_split(torch, kind, n):
    ns = NSTATES[n]
    kw = dict(KINDS[kind], nx=n, ny=n, nt=ns * 4 + 1)
    oc, gp, gpe = pair(precision=atm.FP32, sweep_kernel=atm.SWEEP_PERSISTENT, **kw)
    _, _, gsp = pair(precision=atm.FP32, sweep_kernel=atm.SWEEP_SPLIT, **kw)
    pe, sp = atm.Solver(gp, gpe), atm.Solver(gp, gsp)
    cfg = pe.sweep_config(0)
    assert cfg["kernel"] == "persistent", cfg
    assert ns > cfg["chunk"] > 0, cfg          # several states per cluster
    x = I.uniform_field((ns, n, n), 17, -1.0, 1.0)
    sample = np.unique(np.r_[0, 1, cfg["chunk"] - 1, cfg["chunk"], cfg["chunk"] + 1, ns - 1,
                             np.random.default_rng(n).integers(0, ns, 6)])
    for level in range(len(kw["m"]) + 1):
        tol = fp32_tol(kw, level)
        got = pe.apply_propagator(level, dev(torch, x)).cpu().numpy()
        ref = sp.apply_propagator(level, dev(torch, x)).cpu().numpy()
        want = oracle.apply_prop(oc, level, x[sample])
        for i, j in enumerate(sample):
            ef, es = rel_l2(got[j], want[i]), rel_l2(ref[j], want[i])
            assert ef <= tol and es <= tol, (level, j, ef, es, tol)
            assert ef <= 2 * es + 1e-6, (level, j, ef, es)
        # every state, against the split kernels (both FP32, same operations)
        for j in range(ns):
            assert rel_l2(got[j], ref[j]) <= 2 * tol, (level, j)
    pe.close()
    sp.close()


@pytest.mark.parametrize("n", [64, 256])
def test_persistent_fp32_solve_and_residual_norms(torch, n):
    """An FP32 solve on persistent kernels (residual partial sums per state
    and CTA) has the residual history of the split kernels to FP32 rounding
    and reaches the FP64 sequential solution within the FP32 bar."""
    kw = dict(kind="ac", nx=n, ny=n, dt=1e-4, nt=513 if n == 256 else 2049, m=(4, 4), k=4, nu=1, tol=0.0,
              max_iter=4, precision=atm.FP32)
    u0 = I.uniform_field((n, n), 18)
    out = {}
    for sk in (atm.SWEEP_PERSISTENT, atm.SWEEP_SPLIT):
        oc, gp, gs = pair(sweep_kernel=sk, **kw)
        s = atm.Solver(gp, gs)
        s.set_initial_condition(dev(torch, u0))
        s.solve()
        out[sk] = (s.solution().cpu().numpy(), s.residual_history())
        s.close()
    np.testing.assert_allclose(out[atm.SWEEP_PERSISTENT][1], out[atm.SWEEP_SPLIT][1], rtol=1e-3)
    assert rel_l2(out[atm.SWEEP_PERSISTENT][0], out[atm.SWEEP_SPLIT][0]) <= 1e-5
    want = np.zeros_like(out[atm.SWEEP_SPLIT][0])
    want[0] = u0
    oracle.solve(oc, want, 4, 0.0)
    assert rel_l2(out[atm.SWEEP_PERSISTENT][0], want) <= 1e-4


@pytest.mark.parametrize("cpo", [False, True])
def test_persistent_inner_cycles_of_the_refined_mode(torch, cpo):
    """Increments around a base (the base rows staged in the second tile) in
    the refined mode's FP32 inner cycles: the FP64 fixed point within 1e-7."""
    kw = dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=2049, m=(8, 4), k=4, nu=1, tol=1e-8, max_iter=60,
              precision=atm.FP32_REFINED, sweep_kernel=atm.SWEEP_PERSISTENT, cpoint_only=cpo)
    oc, gp, gs = pair(**kw)
    s = atm.Solver(gp, gs)
    assert s.sweep_config(0)["kernel"] == "persistent"
    u0 = I.uniform_field((128, 128), 19)
    s.set_initial_condition(dev(torch, u0))
    r = s.solve()
    assert r["converged"], r
    seq = oracle.sequential(oc, u0)
    m0 = kw["m"][0]
    got = np.stack([s.solution(t, 1).cpu().numpy()[0] for t in range(0, kw["nt"], m0)])
    assert rel_l2(got, seq[::m0]) <= 1e-7
    s.close()
