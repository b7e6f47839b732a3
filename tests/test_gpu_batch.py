"""Device-side convergence loop (one graph launch per solve, conditional WHILE
node) and batched solves of independent problems in one graph launch, both
against the host-driven solve: identical arithmetic, so identical iterates and
residual histories bit for bit."""
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


def make(torch, kw, seed, use_graph):
    oc, gp, gs = pair(use_graph=use_graph, **kw)
    s = atm.Solver(gp, gs)
    shape = s.state_shape
    u0 = I.heat1d_initial_condition(kw["nx"], seed) if kw["kind"] == "heat1d" else I.uniform_field(shape, seed)
    s.set_initial_condition(torch.as_tensor(u0, device="cuda:0"))
    return oc, s, u0


CASES = [
    dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=257, m=(4, 4), k=3, nu=1, tol=1e-9, max_iter=60),
    dict(kind="heat2d", nx=128, ny=64, dt=1e-3, nt=513, m=(8,), k=4, nu=0, tol=1e-10, max_iter=60),
    dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=513, m=(8, 4), k=4, nu=1, tol=1e-8, max_iter=60,
         precision=atm.FP32),
    dict(kind="heat1d", nx=127, dt=1 / 1024, nt=1025, m=(8,), k=4, nu=1, tol=1e-10, max_iter=60),
    dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=300, m=(4, 2, 2), k=5, nu=1, tol=1e-9, max_iter=60,
         algorithm="mgrit"),
    dict(kind="heat2d", nx=64, ny=64, dt=1e-3, nt=257, m=(16,), k=2, nu=1, tol=1e-30, max_iter=3),
    dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9, max_iter=40,
         precision=atm.FP32_REFINED),
    dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9, max_iter=40,
         precision=atm.FP32_REFINED, cpoint_only=True),
    dict(kind="heat1d", nx=127, dt=1 / 1024, nt=1025, m=(8,), k=4, nu=1, tol=1e-10, max_iter=40,
         precision=atm.FP32_REFINED, cpoint_only=True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_device_loop_equals_host_loop(torch, case):
    kw = CASES[case]
    _, a, _ = make(torch, kw, 3, 1)
    _, b, _ = make(torch, kw, 3, 2)
    ra, rb = a.solve(), b.solve()
    assert ra["iterations"] == rb["iterations"]
    np.testing.assert_array_equal(a.residual_history(), b.residual_history())
    np.testing.assert_array_equal(a.solution().cpu().numpy(), b.solution().cpu().numpy())


def test_batch_equals_individual_solves(torch):
    singles, batch = [], []
    for i, kw in enumerate(CASES):
        _, s, _ = make(torch, kw, 10 + i, 1)
        singles.append((s, s.solve()))
        _, b, _ = make(torch, kw, 10 + i, 1)
        batch.append(b)
    res = atm.batch_solve(batch)
    for (s, rs), b, rb in zip(singles, batch, res):
        assert rs["iterations"] == rb["iterations"]
        np.testing.assert_array_equal(s.residual_history(), b.residual_history())
        np.testing.assert_array_equal(s.solution().cpu().numpy(), b.solution().cpu().numpy())
    # the converged FP64 Allen-Cahn member equals the oracle's sequential solution
    oc, _, _ = pair(**CASES[0])
    seq = oracle.sequential(oc, I.uniform_field((64, 64), 10))
    assert rel_l2(batch[0].solution().cpu().numpy(), seq) <= 1e-8


def test_batch_rejects_unsupported_handles(torch):
    oc, gp, gs = pair(kind="ac", nx=64, ny=64, dt=1e-4, nt=129, m=(4,), algorithm="seq")
    s = atm.Solver(gp, gs)
    with pytest.raises(atm.AtmError, match="UNSUPPORTED"):
        atm.batch_solve([s])
