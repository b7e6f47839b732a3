"""atm_apply_propagator_noalloc, the entry point for callers that may not
allocate device memory (its scratch lives in a static device array of the
library), against the regular workspace-based atm_apply_propagator and against
the FP64 oracle.

Kept in a file that pytest collects last.  Runs alone in a fresh process as
well as after the other tests: the first call on the device performs the
library's one-time symbol lookup itself."""
import ctypes

import numpy as np
import pytest

import atm_inputs as I
import oracle
import paper_2107_09596_gb300 as atm
from helpers import pair, rel_l2

pytestmark = pytest.mark.gpu


def _noalloc(lib, prob, desc, level, x, out, stream):
    return lib.atm_apply_propagator_noalloc(ctypes.byref(prob), ctypes.byref(desc), level,
                                            ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), x.shape[0],
                                            ctypes.c_void_p(stream.cuda_stream))


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    atm._build.build()
    atm.load()
    return torch


def test_noalloc_matches_apply_propagator_on_two_calls(torch):
    lib = atm.load()
    prob = atm.make_problem(atm.ALLEN_CAHN, 256, 256, dt=1e-4, nt_points=4097, eps=0.02)
    desc = atm.make_solver(atm.AT_MGRIT, m=(16, 16), k=8, nu=1, precision=atm.FP64)
    ref = atm.Solver(prob, desc)
    stream = torch.cuda.current_stream()
    # two calls in a row on different levels and inputs; each must equal the
    # regular entry point within the FP64 propagator tolerance of the suite
    for level, seed in ((0, 21), (2, 22)):
        x = torch.as_tensor(I.uniform_field((16, 256, 256), seed, -1.0, 1.0), device="cuda:0")
        want = ref.apply_propagator(level, x).cpu().numpy()
        got = torch.full_like(x, float("nan"))
        st = _noalloc(lib, prob, desc, level, x, got, stream)
        assert st == 0, lib.atm_last_error().decode()
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        for s in range(x.shape[0]):
            rel = np.linalg.norm(g[s] - want[s]) / np.linalg.norm(want[s])
            assert rel <= 1e-13, (level, s, rel)
    ref.close()


def test_noalloc_matches_the_oracle_in_place(torch):
    """Every level of a three-level Allen-Cahn hierarchy (PR-ADI fine step,
    split-BE coarse steps with the exact reaction flow) on a 128 x 64 grid,
    with in == out, against the oracle's propagators; two calls in a row."""
    lib = atm.load()
    oc, gp, gs = pair(kind="ac", nx=128, ny=64, lx=1.0, ly=0.5, dt=1e-4, nt=257, m=(4, 4), k=3)
    stream = torch.cuda.current_stream()
    for rep in range(2):
        for level in range(3):
            x = I.uniform_field((7, 64, 128), 30 + 3 * rep + level, -1.0, 1.0)
            want = oracle.apply_prop(oc, level, x)
            buf = torch.as_tensor(x, device="cuda:0")
            st = _noalloc(lib, gp, gs, level, buf, buf, stream)
            assert st == 0, lib.atm_last_error().decode()
            torch.cuda.synchronize()
            got = buf.cpu().numpy()
            for s in range(x.shape[0]):
                assert rel_l2(got[s], want[s]) <= 1e-13, (rep, level, s, rel_l2(got[s], want[s]))


def test_noalloc_learned_description(torch):
    """A learned coarse propagator description: level 2 runs (split-BE, as the
    handle would), level 1 is rejected with a message naming the network."""
    lib = atm.load()
    oc, gp, gs = pair(kind="ac", nx=64, ny=64, dt=1e-4, nt=257, m=(4, 4), k=3)
    gs.coarse_prop = atm.PROP_LEARNED
    stream = torch.cuda.current_stream()
    x = I.uniform_field((3, 64, 64), 40, -1.0, 1.0)
    buf = torch.as_tensor(x, device="cuda:0")
    out = torch.empty_like(buf)
    st = _noalloc(lib, gp, gs, 2, buf, out, stream)
    assert st == 0, lib.atm_last_error().decode()
    torch.cuda.synchronize()
    want = oracle.apply_prop(oc, 2, x)
    assert rel_l2(out.cpu().numpy(), want) <= 1e-13
    st = _noalloc(lib, gp, gs, 1, buf, out, stream)
    assert atm.STATUS[st] == "ATM_ERR_UNSUPPORTED"
    assert "learned" in lib.atm_last_error().decode()


def test_noalloc_rejects_requests_beyond_its_limit(torch):
    lib = atm.load()
    stream = torch.cuda.current_stream()
    prob = atm.make_problem(atm.HEAT2D, 512, 512, dt=1e-4, nt_points=65)
    desc = atm.make_solver(atm.AT_MGRIT, m=(4,), k=2, precision=atm.FP64)
    x = torch.zeros((17, 512, 512), dtype=torch.float64, device="cuda:0")   # 34 MiB > 32 MiB
    out = torch.empty_like(x)
    st = _noalloc(lib, prob, desc, 0, x, out, stream)
    assert atm.STATUS[st] == "ATM_ERR_INVALID_ARG"
    assert "limit" in lib.atm_last_error().decode()
    st = _noalloc(lib, prob, desc, 0, x[:16], out[:16], stream)      # exactly 32 MiB
    assert st == 0, lib.atm_last_error().decode()
    torch.cuda.synchronize()
    assert torch.all(out[:16] == 0)     # Phi(0) = 0
