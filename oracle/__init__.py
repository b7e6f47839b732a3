"""CPU oracle for AT-MGRIT (arXiv 2107.09596) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2107_09596_gb300``)
never imports it, and it never imports the product package.

``atm_oracle.c`` is plain FP64 C (built with ``-ffp-contract=off``) and
``theory.py`` holds the paper's closed forms (Sec. 3) in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "atm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HEAT1D, HEAT2D, ALLEN_CAHN, GRAY_SCOTT = 0, 1, 2, 3
PROP_SPLIT, PROP_PR, PROP_FINEPOW = 0, 1, 2
MAXLEV = 8


class OrCfg(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("lx", ctypes.c_double),
        ("ly", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("nt", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("levels", ctypes.c_int),
        ("m", ctypes.c_int * MAXLEV),
        ("k", ctypes.c_int),
        ("nu", ctypes.c_int),
        ("prop", ctypes.c_int * MAXLEV),
        ("react_sub", ctypes.c_int * MAXLEV),
        ("react_exact", ctypes.c_int * MAXLEV),
        ("fcycle", ctypes.c_int),
        ("ext_prop", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP if available)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and \
                os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"]
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        try:
            subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrCfg)
        dp = ctypes.c_void_p
        L.or_level_points.argtypes = [P, ctypes.c_int]
        L.or_level_points.restype = ctypes.c_int
        L.or_level_dt.argtypes = [P, ctypes.c_int]
        L.or_level_dt.restype = ctypes.c_double
        L.or_apply_prop.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_int]
        L.or_sequential.argtypes = [P, dp, dp]
        L.or_solve.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_double, dp]
        L.or_solve.restype = ctypes.c_int
        L.or_cpoint_residual_norm.argtypes = [P, dp, dp]
        L.or_cpoint_residual_norm.restype = ctypes.c_double
        L.or_nested_guess.argtypes = [P, dp]
        L.or_nested_guess.restype = None
        L.or_full_residual_norm.argtypes = [P, dp, dp]
        L.or_full_residual_norm.restype = ctypes.c_double
        L.or_frelax_level.argtypes = [P, ctypes.c_int, dp, dp]
        L.or_crelax_level.argtypes = [P, ctypes.c_int, dp, dp]
        L.or_restrict_level.argtypes = [P, ctypes.c_int, dp, dp, dp, dp, dp]
        L.or_coarsest_level.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# Gray-Scott propagators and their C callbacks stay alive for the process
_keep = []


def make_cfg(kind, nx, ny=1, lx=1.0, ly=1.0, dt=1.0 / 1024, nt=1025, eps=0.02,
             m=(8,), k=4, nu=1, prop=None, react_sub=None, react_exact=None, fcycle=False,
             gs=None) -> OrCfg:
    """Problem + solver description.  ``m`` has one entry per coarsening
    (levels = len(m) + 1).  ``k <= 0`` selects plain MGRIT.  ``prop`` per level
    defaults to PR on level 0 and split-BE on coarser levels (2D) or BE (1D).
    Gray-Scott (Sec. 5.1): ``gs`` = dict(du, dv, feed, kill, tol, max_iter);
    the propagator object is ``cfg.gray_scott``."""
    c = OrCfg()
    if kind == GRAY_SCOTT:
        from .gray_scott import GrayScott, make_callback
        p = dict(du=8e-5, dv=4e-5, feed=0.024, kill=0.06, tol=1e-10, max_iter=50)
        p.update(gs or {})
        model = GrayScott(nx, ny, lx, ly, **p)
        cb = make_callback(model)
        _keep.append((model, cb))
        c.ext_prop = ctypes.cast(cb, ctypes.c_void_p).value
        c.gray_scott = model
    c.kind, c.nx, c.ny = kind, nx, (1 if kind == HEAT1D else ny)
    c.lx, c.ly, c.dt, c.nt, c.eps = lx, ly, dt, nt, eps
    c.levels = len(m) + 1
    for i, mi in enumerate(m):
        c.m[i] = mi
    c.k, c.nu = k, nu
    c.fcycle = int(fcycle)
    if prop is None:
        prop = [PROP_PR if (kind != HEAT1D and l == 0) else PROP_SPLIT for l in range(c.levels)]
    for i, p in enumerate(prop):
        c.prop[i] = p
    if react_sub is not None:
        for i, s in enumerate(react_sub):
            c.react_sub[i] = s
    if react_exact is not None:
        for i, e in enumerate(react_exact):
            c.react_exact[i] = int(e)
    return c


def state_shape(c: OrCfg):
    if c.kind == GRAY_SCOTT:
        return (2, c.ny, c.nx)
    return (c.nx,) if c.kind == HEAT1D else (c.ny, c.nx)


def level_points(c: OrCfg, l: int) -> int:
    return lib().or_level_points(ctypes.byref(c), l)


def level_dt(c: OrCfg, l: int) -> float:
    return lib().or_level_dt(ctypes.byref(c), l)


def apply_prop(c: OrCfg, l: int, states: np.ndarray) -> np.ndarray:
    """Phi_l applied to each state of ``states`` (shape (S,) + state_shape)."""
    x = np.ascontiguousarray(states, dtype=np.float64)
    out = np.empty_like(x)
    ns = x.shape[0]
    lib().or_apply_prop(ctypes.byref(c), l, _ptr(x), _ptr(out), ns)
    return out


def sequential(c: OrCfg, u0: np.ndarray, g: np.ndarray | None = None) -> np.ndarray:
    """Sequential time stepping (Sec. 2): all nt states from u0."""
    u = np.zeros((c.nt,) + state_shape(c), dtype=np.float64)
    u[0] = u0
    lib().or_sequential(ctypes.byref(c), _ptr(g), _ptr(u))
    return u


def solve(c: OrCfg, u: np.ndarray, max_iter: int, tol: float = 0.0,
          g: np.ndarray | None = None):
    """Run AT-MGRIT/MGRIT on the iterate ``u`` (modified in place: u[0] is the
    initial condition, the rest the initial guess).  Returns (iterations,
    residual history of length iterations + 1)."""
    assert u.dtype == np.float64 and u.flags["C_CONTIGUOUS"]
    hist = np.zeros(max_iter + 1)
    it = lib().or_solve(ctypes.byref(c), _ptr(g), _ptr(u), max_iter, tol, _ptr(hist))
    if it < 0:
        raise ValueError("invalid oracle configuration")
    return it, hist[: it + 1].copy()


def nested_guess(c: OrCfg, u: np.ndarray) -> None:
    """Nested iteration: overwrite the level-0 C-points i >= 1 of ``u`` with the
    coarse hierarchy's values (coarsest level stepped sequentially, injection
    and F-relaxation on each finer coarse level)."""
    assert u.dtype == np.float64 and u.flags["C_CONTIGUOUS"]
    lib().or_nested_guess(ctypes.byref(c), _ptr(u))


def cpoint_residual_norm(c: OrCfg, u: np.ndarray, g=None) -> float:
    return lib().or_cpoint_residual_norm(ctypes.byref(c), _ptr(g), _ptr(u))


def full_residual_norm(c: OrCfg, u: np.ndarray, g=None) -> float:
    return lib().or_full_residual_norm(ctypes.byref(c), _ptr(g), _ptr(u))


def frelax_level(c: OrCfg, l: int, u: np.ndarray, g=None) -> None:
    lib().or_frelax_level(ctypes.byref(c), l, _ptr(g), _ptr(u))


def crelax_level(c: OrCfg, l: int, u: np.ndarray, g=None) -> None:
    lib().or_crelax_level(ctypes.byref(c), l, _ptr(g), _ptr(u))


def restrict_level(c: OrCfg, l: int, u: np.ndarray, g=None):
    """Residual, injection and FAS right-hand side for level l+1: (v, r, gc)."""
    nc = level_points(c, l + 1)
    shp = (nc,) + state_shape(c)
    v, r, gc = np.zeros(shp), np.zeros(shp), np.zeros(shp)
    lib().or_restrict_level(ctypes.byref(c), l, _ptr(g), _ptr(u), _ptr(v), _ptr(r), _ptr(gc))
    return v, r, gc


def coarsest_level(c: OrCfg, l: int, v, r, gc) -> np.ndarray:
    u = np.zeros_like(v)
    lib().or_coarsest_level(ctypes.byref(c), l, _ptr(v), _ptr(r), _ptr(gc), _ptr(u))
    return u


def num_threads() -> int:
    return lib().or_num_threads()


def local_grid(p: int, k: int):
    """Index set of the p-th local coarse grid (Sec. 2.1): [max(0, p-k+1), p]."""
    return list(range(max(0, p - k + 1), p + 1))
