"""C-point storage on level 0 (Sec. 2.1: an iterate's F-points are the
F-relaxation of its C-points, so only the C-points and one working state per
interval are kept).  The cycle performs the same arithmetic on the same
values as with full storage, so iterates, residual histories and every
recomputed F-point agree bit for bit; the refined mode with C-point storage
takes its FP64 residual at the C-points and must reach the FP64 fixed point
(the oracle's sequential solution) within 1e-7."""
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


def field(kw, seed):
    if kw["kind"] == "heat1d":
        return I.heat1d_initial_condition(kw["nx"], seed)
    return I.uniform_field((kw.get("ny", 1), kw["nx"]), seed)


def run(torch, kw, cpo, seed=0, guess=None):
    oc, gp, gs = pair(cpoint_only=cpo, **kw)
    s = atm.Solver(gp, gs)
    s.set_initial_condition(torch.as_tensor(field(kw, seed), device="cuda:0"))
    if guess is not None:
        s.set_initial_guess(guess)
    r = s.solve()
    return oc, s, r


CASES = {
    "ac_fcf_ragged": dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=300, m=(4, 4), k=3, nu=1, tol=1e-9, max_iter=40),
    "ac_f_4lvl": dict(kind="ac", nx=32, ny=32, dt=1e-4, nt=257, m=(4, 2, 2), k=4, nu=0, tol=1e-9, max_iter=40),
    "heat2d_mgrit": dict(kind="heat2d", nx=64, ny=128, dt=1e-3, nt=513, m=(8,), k=4, nu=1, tol=1e-10,
                         max_iter=40, algorithm="mgrit"),
    "heat1d_ragged": dict(kind="heat1d", nx=127, dt=1 / 1024, nt=1000, m=(8,), k=4, nu=1, tol=1e-10, max_iter=60),
    # FP32 results depend on the kernel (chunking of the line recurrences): both
    # storages get the same fixed kernel instead of their own autotuned pick
    "ac_fp32": dict(kind="ac", nx=128, ny=128, dt=1e-4, nt=513, m=(8, 4), k=4, nu=1, tol=1e-5, max_iter=40,
                    precision=atm.FP32, sweep_kernel=atm.SWEEP_FUSED),
    "ac_seq": dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=300, m=(16,), algorithm="seq"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_cpoint_storage_equals_full_storage(torch, case):
    kw = CASES[case]
    _, full, rf = run(torch, kw, False, seed=4)
    _, cpo, rc = run(torch, kw, True, seed=4)
    assert rf["iterations"] == rc["iterations"]
    np.testing.assert_array_equal(full.residual_history(), cpo.residual_history())
    np.testing.assert_array_equal(full.solution().cpu().numpy(), cpo.solution().cpu().numpy())
    assert atm.workspace_size(cpo.problem, cpo.desc) < atm.workspace_size(full.problem, full.desc)


def test_cpoint_storage_partial_reads_and_host_buffers(torch):
    kw = CASES["ac_fcf_ragged"]
    _, full, _ = run(torch, kw, False, seed=5)
    _, cpo, _ = run(torch, kw, True, seed=5)
    want = full.solution().cpu().numpy()
    for t0, count in [(0, 1), (3, 1), (5, 11), (13, 40), (255, 45), (299, 1), (290, 10)]:
        got = cpo.solution(t0, count).cpu().numpy()
        np.testing.assert_array_equal(got, want[t0:t0 + count])
    host = np.empty((17,) + cpo.state_shape)
    cpo.solution(101, 17, out=host)
    np.testing.assert_array_equal(host, want[101:118])


def test_cpoint_storage_matches_the_oracle_iterates(torch):
    kw = dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=137, m=(4, 3), k=3, nu=1, max_iter=2)
    oc, s, _ = run(torch, kw, True, seed=2)
    want = np.zeros((kw["nt"], 64, 64))
    want[0] = field(kw, 2)
    _, hist = oracle.solve(oc, want, 2, 0.0)
    assert rel_l2(s.solution().cpu().numpy(), want) <= 1e-12
    np.testing.assert_allclose(s.residual_history(), hist, rtol=1e-11)


def test_cpoint_storage_keeps_only_cpoints_of_a_guess(torch):
    """Only the C-points of an initial guess act (the first F-relaxation
    overwrites the rest): full and C-point storage agree for a random guess."""
    kw = dict(CASES["ac_fcf_ragged"], max_iter=3, tol=0.0)
    g = torch.as_tensor(I.random_guess(kw["nt"], (64, 64), 9), device="cuda:0")
    _, full, _ = run(torch, kw, False, seed=6, guess=g)
    _, cpo, _ = run(torch, kw, True, seed=6, guess=g)
    np.testing.assert_array_equal(full.residual_history(), cpo.residual_history())
    np.testing.assert_array_equal(full.solution().cpu().numpy(), cpo.solution().cpu().numpy())


@pytest.mark.parametrize("case", ["ac", "heat1d"])
def test_refined_with_cpoint_storage_reaches_fp64_accuracy(torch, case):
    if case == "ac":
        kw = dict(kind="ac", nx=64, ny=64, dt=1e-4, nt=257, m=(4, 4), k=4, nu=1, tol=1e-9)
    else:
        kw = dict(kind="heat1d", nx=127, dt=1 / 1024, nt=1025, m=(8,), k=4, nu=1, tol=1e-10)
    oc, s, r = run(torch, dict(kw, max_iter=80, precision=atm.FP32_REFINED), True, seed=7)
    _, s64, r64 = run(torch, dict(kw, max_iter=80), False, seed=7)
    assert r["converged"] and r64["converged"], (r, r64)
    seq = oracle.sequential(oc, field(kw, 7))
    err = rel_l2(s.solution().cpu().numpy(), seq)
    assert err <= 1e-7, err
    assert r["iterations"] <= r64["iterations"] + 3, (r, r64)
    # the history is the FP64 C-point residual of the iterate: recompute its last entry
    u = s.solution().cpu().numpy()
    cp = oracle.cpoint_residual_norm(oc, np.ascontiguousarray(u))
    floor = 4 * 2.2e-16 * np.sqrt(u.size) * np.abs(u).max()   # FP64 rounding of a residual evaluation
    assert abs(cp - s.residual_history()[-1]) <= 1e-3 * cp + floor
