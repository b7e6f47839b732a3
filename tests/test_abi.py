"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function declared in include/atm.h, and validates problem/solver
descriptions on the host (atm_workspace_size touches no device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def atm():
    import paper_2107_09596_gb300 as atm
    atm._build.build()
    atm.load()
    return atm


def declared_functions():
    text = open(os.path.join(ROOT, "include", "atm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(atm_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    import paper_2107_09596_gb300 as atm
    assert set(declared_functions()) == set(atm.EXPORTS)


def test_library_exports_every_declared_symbol(atm):
    lib = ctypes.CDLL(atm.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_workspace_size_cfg2_and_validation(atm):
    p = atm.make_problem(atm.ALLEN_CAHN, 256, 256, dt=1e-4, nt_points=4097, eps=0.02)
    s = atm.make_solver(atm.AT_MGRIT, m=(16, 16), k=8, nu=1, tol=1e-8, precision=atm.FP64)
    n = atm.workspace_size(p, s)
    state = 256 * 256 * 8
    # level 0 (4097) + C-relaxation values (257) + 4 arrays on levels 1 (257) and 2 (17)
    assert n >= (4097 + 257 + 4 * 257 + 4 * 17) * state
    assert n < (4097 + 257 + 4 * 257 + 4 * 17 + 300) * state
    s32 = atm.make_solver(atm.AT_MGRIT, m=(16, 16), k=8, nu=1, precision=atm.FP32)
    assert atm.workspace_size(p, s32) < 0.6 * n


@pytest.mark.parametrize("change, status", [
    (dict(nx=100), "ATM_ERR_INVALID_ARG"),          # 2D grid not a power of two
    (dict(nt_points=1), "ATM_ERR_INVALID_ARG"),
    (dict(dt=0.0), "ATM_ERR_INVALID_ARG"),
])
def test_invalid_problem_rejected(atm, change, status):
    kw = dict(kind=atm.ALLEN_CAHN, nx=64, ny=64, dt=1e-4, nt_points=129, eps=0.02)
    kw.update(change)
    p = atm.make_problem(**kw)
    s = atm.make_solver(atm.AT_MGRIT, m=(4, 4), k=3)
    with pytest.raises(atm.AtmError) as e:
        atm.workspace_size(p, s)
    assert status in str(e.value)


@pytest.mark.parametrize("change", [dict(m=(1,)), dict(k=0), dict(nu=3), dict(m=(64, 64))])
def test_invalid_solver_rejected(atm, change):
    p = atm.make_problem(atm.HEAT1D, 127, dt=1 / 1024, nt_points=1025)
    kw = dict(algorithm=atm.AT_MGRIT, m=(8,), k=4, nu=1)
    kw.update(change)
    s = atm.make_solver(**kw)
    with pytest.raises(atm.AtmError):
        atm.workspace_size(p, s)
