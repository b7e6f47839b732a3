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
    names = re.findall(r"\b(atm_[a-z0-9_]+)\s*\(", text)
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


@pytest.mark.parametrize("change", [dict(m=(1,)), dict(k=0), dict(nu=3), dict(m=(64, 64)),
                                    dict(inner_coarse_relax=2), dict(inner_coarse_relax=-1)])
def test_invalid_solver_rejected(atm, change):
    p = atm.make_problem(atm.HEAT1D, 127, dt=1 / 1024, nt_points=1025)
    kw = dict(algorithm=atm.AT_MGRIT, m=(8,), k=4, nu=1)
    kw.update(change)
    s = atm.make_solver(**kw)
    with pytest.raises(atm.AtmError):
        atm.workspace_size(p, s)


def test_gray_scott_workspace_and_validation(atm):
    # 128^2 x 16384 points, m = 64, full storage: level 0, four arrays on level 1,
    # and the Newton kernel's slices (two per SM: five FP64 and 23 FP32 vectors)
    p = atm.make_problem(atm.GRAY_SCOTT, 128, 128, lx=2.5, ly=2.5, dt=256 / 16383, nt_points=16384)
    s = atm.make_solver(atm.AT_MGRIT, m=(64,), k=128, nu=0, tol=1e-7)
    n = atm.workspace_size(p, s)
    state = 2 * 128 * 128 * 8
    slices = 2 * 152 * (5 * state + 23 * state // 2)
    base = (16384 + 4 * 256) * state
    assert base + slices <= n < base + slices + 300 * state
    # C-point storage keeps the C-points and one working state per interval
    sc = atm.make_solver(atm.AT_MGRIT, m=(64,), k=128, nu=0, tol=1e-7, cpoint_only=True)
    assert atm.workspace_size(p, sc) < n - 15000 * state
    for change in (dict(precision=atm.FP32), dict(precision=atm.FP32_REFINED),
                   dict(sweep_kernel=atm.SWEEP_FUSED), dict(sweep_kernel=atm.SWEEP_CHAIN),
                   dict(coarse_prop=atm.PROP_LEARNED)):
        bad = atm.make_solver(atm.AT_MGRIT, m=(64,), k=128, nu=0, **change)
        with pytest.raises(atm.AtmError):
            atm.workspace_size(p, bad)
    for change in (dict(nx=4), dict(ny=1024), dict(du=-1.0), dict(newton_max_iter=501)):
        kw = dict(kind=atm.GRAY_SCOTT, nx=64, ny=64, lx=2.5, ly=2.5, dt=0.01, nt_points=129)
        kw.update(change)
        with pytest.raises(atm.AtmError):
            atm.workspace_size(atm.make_problem(**kw), atm.make_solver(atm.AT_MGRIT, m=(8,), k=4))
    # any grid size from 8 to 512 is allowed
    atm.workspace_size(atm.make_problem(atm.GRAY_SCOTT, 40, 24, lx=2.5, ly=1.5, dt=0.01, nt_points=65),
                       atm.make_solver(atm.MGRIT, m=(8,), k=1))


def test_tune_cache_round_trip_and_malformed_text(atm):
    """The autotuner's choices as text (no device work): an imported line is
    exported again; malformed text is rejected and imports nothing."""
    before = atm.tune_cache_export()
    atm.tune_cache_import("testkey d0 T4\t0,1,-1,2\n")
    out = atm.tune_cache_export()
    assert "testkey d0 T4\t0,1,-1,2\n" in out
    for bad in ("no tab here\n", "\t1,2\n", "k\t1,x\n"):
        with pytest.raises(atm.AtmError):
            atm.tune_cache_import(bad)
    assert atm.tune_cache_export() == out
    assert set(before.splitlines()) <= set(out.splitlines())
