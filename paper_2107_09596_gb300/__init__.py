"""GB300 (sm_103a) AT-MGRIT space-time sweep (arXiv 2107.09596).

Thin ctypes binding over ``libatm.so`` (``include/atm.h``): argument
marshalling only.  Every step of the sweep runs in the library's CUDA kernels;
there is no CPU fallback -- importing the binding without the built library on
a machine raises.  PyTorch provides device memory (the workspace and state
buffers) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HEAT1D, HEAT2D, ALLEN_CAHN, GRAY_SCOTT = 0, 1, 2, 3
PROP_SPLIT_BE, PROP_PR_ADI, PROP_LEARNED, PROP_LEARNED_CORRECTION = 0, 1, 2, 3
REACT_EXACT, REACT_SUBSTEPS = 0, 1
SEQUENTIAL, MGRIT, AT_MGRIT = 0, 1, 2
FP64, FP32, FP32_REFINED, FP64_FF, FP32_REFINED_FF = 0, 1, 2, 3, 4
SWEEP_AUTO, SWEEP_SPLIT, SWEEP_FUSED, SWEEP_CHAIN, SWEEP_PERSISTENT = 0, 1, 2, 3, 4
STAGE_F_RELAX, STAGE_C_RELAX, STAGE_RESTRICT, STAGE_COARSEST, STAGE_CORRECT = range(5)
ARRAY_U, ARRAY_V, ARRAY_R, ARRAY_G = range(4)
MAX_LEVELS = 8

STATUS = {0: "ATM_OK", 1: "ATM_ERR_INVALID_ARG", 2: "ATM_ERR_CUDA", 3: "ATM_ERR_OOM",
          4: "ATM_ERR_NOT_CONVERGED", 5: "ATM_ERR_DIVERGED", 6: "ATM_ERR_TIMEOUT",
          7: "ATM_ERR_UNSUPPORTED"}


class AtmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("dt", ctypes.c_double),
                ("nt_points", ctypes.c_int), ("eps", ctypes.c_double),
                ("gs_du", ctypes.c_double), ("gs_dv", ctypes.c_double),
                ("gs_feed", ctypes.c_double), ("gs_kill", ctypes.c_double),
                ("newton_tol", ctypes.c_double), ("newton_max_iter", ctypes.c_int)]


class SolverDesc(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int), ("levels", ctypes.c_int),
                ("m", ctypes.c_int * MAX_LEVELS), ("k", ctypes.c_int), ("nu", ctypes.c_int),
                ("fine_prop", ctypes.c_int), ("coarse_prop", ctypes.c_int),
                ("reaction_substeps", ctypes.c_int * MAX_LEVELS),
                ("coarse_reaction", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("sweep_kernel", ctypes.c_int),
                ("refine_inner_cycles", ctypes.c_int), ("cycle_type", ctypes.c_int), ("forcing", ctypes.c_int),
                ("nested_iteration", ctypes.c_int),
                ("cpoint_storage_only", ctypes.c_int), ("refine_coarse_relax", ctypes.c_int)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("log_every", ctypes.c_int), ("h_loss_history", ctypes.c_void_p),
                ("history_cap", ctypes.c_int)]


class TrainResult(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("logged", ctypes.c_int), ("final_loss", ctypes.c_double),
                ("time_ms", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("initial_residual", ctypes.c_double), ("final_residual", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("fallback", ctypes.c_int),
                ("fallback_iterations", ctypes.c_int), ("fallback_residual", ctypes.c_double)]


EXPORTS = ["atm_workspace_size", "atm_create", "atm_set_initial_condition",
           "atm_set_initial_guess", "atm_solve", "atm_get_solution",
           "atm_get_residual_history", "atm_apply_propagator", "atm_run_stage",
           "atm_level_read", "atm_level_write", "atm_level_points",
           "atm_last_launch_count", "atm_get_kernel_profile", "atm_apply_propagator_noalloc",
           "atm_nn_param_count", "atm_nn_workspace_size", "atm_nn_apply", "atm_nn_loss_grad",
           "atm_train_learned_coarse", "atm_set_learned_coarse", "atm_batch_solve", "atm_last_error",
           "atm_get_sweep_config", "atm_set_rhs", "atm_get_newton_stats", "atm_measure_fp64_rate",
           "atm_tune_cache_export", "atm_tune_cache_import", "atm_destroy"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libatm.so (building it with nvcc if absent and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing: run paper_2107_09596_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.atm_workspace_size.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(SolverDesc), ctypes.POINTER(ctypes.c_size_t)]
    L.atm_create.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(SolverDesc), vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.atm_set_initial_condition.argtypes = [vp, vp]
    L.atm_set_initial_guess.argtypes = [vp, vp]
    L.atm_set_rhs.argtypes = [vp, vp]
    L.atm_solve.argtypes = [vp, ctypes.POINTER(Result)]
    L.atm_get_solution.argtypes = [vp, i, i, vp]
    L.atm_get_residual_history.argtypes = [vp, vp, i, ctypes.POINTER(i)]
    L.atm_apply_propagator.argtypes = [vp, i, vp, vp, i]
    L.atm_run_stage.argtypes = [vp, i, i]
    L.atm_level_read.argtypes = [vp, i, i, i, i, vp]
    L.atm_level_write.argtypes = [vp, i, i, i, i, vp]
    L.atm_level_points.argtypes = [vp, i]
    L.atm_level_points.restype = i
    L.atm_last_launch_count.argtypes = [vp]
    L.atm_last_launch_count.restype = ctypes.c_longlong
    L.atm_get_kernel_profile.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
    L.atm_get_sweep_config.argtypes = [vp, i, ctypes.POINTER(i)]
    L.atm_get_newton_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.atm_apply_propagator_noalloc.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(SolverDesc), i, vp, vp, i, vp]
    L.atm_nn_param_count.restype = i
    L.atm_nn_workspace_size.argtypes = [i, i, i, i, ctypes.POINTER(ctypes.c_size_t)]
    L.atm_nn_apply.argtypes = [vp, vp, vp, i, i, i, vp, ctypes.c_size_t, vp]
    L.atm_nn_loss_grad.argtypes = [vp, vp, vp, i, i, i, vp, ctypes.POINTER(d), vp, ctypes.c_size_t, vp]
    L.atm_train_learned_coarse.argtypes = [vp, vp, vp, vp, i, i, i, ctypes.POINTER(TrainCfg),
                                           ctypes.POINTER(TrainResult), vp, ctypes.c_size_t, vp]
    L.atm_set_learned_coarse.argtypes = [vp, vp]
    L.atm_batch_solve.argtypes = [ctypes.POINTER(vp), i, vp, ctypes.POINTER(Result)]
    L.atm_measure_fp64_rate.argtypes = [vp, ctypes.POINTER(d)]
    L.atm_tune_cache_export.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.atm_tune_cache_import.argtypes = [ctypes.c_char_p]
    L.atm_last_error.restype = ctypes.c_char_p
    L.atm_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name not in ("atm_level_points", "atm_last_launch_count", "atm_last_error", "atm_destroy",
                        "atm_nn_param_count"):
            getattr(L, name).restype = i
    _lib = L
    return L


def _check(st: int, ok=(0,)):
    if st not in ok:
        raise AtmError(st, load().atm_last_error().decode())
    return st


def make_problem(kind, nx, ny=1, lx=1.0, ly=1.0, dt=1e-3, nt_points=65, eps=0.02,
                 du=8e-5, dv=4e-5, feed=0.024, kill=0.06, newton_tol=1e-10,
                 newton_max_iter=50) -> Problem:
    """Problem description; du, dv, feed, kill and the Newton settings are
    the Gray-Scott parameters (defaults: the values of the paper's Sec. 5.1)."""
    p = Problem()
    p.kind, p.nx, p.ny = kind, nx, ny
    p.lx, p.ly, p.dt, p.nt_points, p.eps = lx, ly, dt, nt_points, eps
    p.gs_du, p.gs_dv, p.gs_feed, p.gs_kill = du, dv, feed, kill
    p.newton_tol, p.newton_max_iter = newton_tol, newton_max_iter
    return p


def make_solver(algorithm=AT_MGRIT, m=(8,), k=4, nu=1, fine_prop=PROP_PR_ADI,
                coarse_prop=PROP_SPLIT_BE, reaction_substeps=None, coarse_reaction=REACT_EXACT,
                tol=1e-10, max_iter=50,
                precision=FP64, use_graph=True, profile=False, cpoint_only=False,
                sweep_kernel=0, inner_cycles=0, nested=False, forcing=False, fcycle=False,
                inner_coarse_relax=0) -> SolverDesc:
    s = SolverDesc()
    s.algorithm = algorithm
    s.levels = len(m) + 1
    for j, mj in enumerate(m):
        s.m[j] = mj
    s.k, s.nu = k, nu
    s.fine_prop, s.coarse_prop = fine_prop, coarse_prop
    s.coarse_reaction = coarse_reaction
    if reaction_substeps:
        for j, v in enumerate(reaction_substeps):
            s.reaction_substeps[j] = v
    s.tol, s.max_iter, s.precision, s.use_graph = tol, max_iter, precision, int(use_graph)
    s.profile = int(profile)
    s.cpoint_storage_only = int(cpoint_only)
    s.sweep_kernel = int(sweep_kernel)
    s.refine_inner_cycles = int(inner_cycles)
    s.nested_iteration = int(nested)
    s.forcing = int(forcing)
    s.cycle_type = int(fcycle)
    s.refine_coarse_relax = int(inner_coarse_relax)
    return s


def workspace_size(problem: Problem, solver: SolverDesc) -> int:
    n = ctypes.c_size_t()
    _check(load().atm_workspace_size(ctypes.byref(problem), ctypes.byref(solver), ctypes.byref(n)))
    return n.value


def measure_fp64_rate(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(load().atm_measure_fp64_rate(ctypes.c_void_p(st.cuda_stream), ctypes.byref(v)))
    return v.value


def tune_cache_export() -> str:
    """The autotuner's kernel choices of this process, as text."""
    n = ctypes.c_size_t()
    _check(load().atm_tune_cache_export(None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().atm_tune_cache_export(buf, n.value, ctypes.byref(n)))
    return buf.value.decode()


def tune_cache_import(text: str) -> None:
    """Add kernel choices exported by tune_cache_export (this or another process)."""
    _check(load().atm_tune_cache_import(text.encode()))


def _ptr(x) -> int:
    """Data pointer of a torch tensor or a numpy array (no copy)."""
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


class Solver:
    """One space-time problem and its solver, living in a torch-allocated workspace."""

    def __init__(self, problem: Problem, solver: SolverDesc, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.problem, self.desc = problem, solver
        self.device = torch.device(device)
        # the library issues all work on its own (non-default) stream, which
        # also allows CUDA-graph capture; calls are ordered against torch's
        # current stream on entry and exit
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        nbytes = workspace_size(problem, solver)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.handle = ctypes.c_void_p()
        self._enter()
        _check(load().atm_create(ctypes.byref(problem), ctypes.byref(solver), ctypes.c_void_p(aligned),
                                 nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.handle)))
        self._leave()
        if problem.kind == GRAY_SCOTT:
            self.state_shape = (2, problem.ny, problem.nx)
        else:
            self.state_shape = (problem.nx,) if problem.kind == HEAT1D else (problem.ny, problem.nx)

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.stream.synchronize()
            load().atm_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f64(self, x):
        """Keep host numpy arrays as they are; make torch tensors contiguous float64."""
        if hasattr(x, "data_ptr"):
            return x.to(dtype=self.torch.float64).contiguous()
        return np.ascontiguousarray(x, dtype=np.float64)

    def set_initial_condition(self, u0):
        u0 = self._f64(u0)
        self._enter()
        _check(load().atm_set_initial_condition(self.handle, ctypes.c_void_p(_ptr(u0))))
        self._leave()
        return u0

    def set_rhs(self, f):
        """Right-hand side f_j (nt states, FP64; state 0 ignored) of a handle created with forcing."""
        f = self._f64(f)
        self._enter()
        _check(load().atm_set_rhs(self.handle, ctypes.c_void_p(_ptr(f))))
        self._leave()
        return f

    def set_initial_guess(self, u=None):
        """Iterate at time points >= 1 from `u` (nt states), or the zero guess."""
        u = None if u is None else self._f64(u)
        self._enter()
        _check(load().atm_set_initial_guess(self.handle, ctypes.c_void_p(None if u is None else _ptr(u))))
        self._leave()
        return u

    def solve(self, allow_not_converged=True) -> dict:
        r = Result()
        ok = (0, 4) if allow_not_converged else (0,)
        self._enter()
        st = _check(load().atm_solve(self.handle, ctypes.byref(r)), ok)
        self._leave()
        return {"status": STATUS[st], "iterations": r.iterations, "converged": bool(r.converged),
                "initial_residual": r.initial_residual, "final_residual": r.final_residual,
                "time_ms": r.time_ms, "launches": load().atm_last_launch_count(self.handle),
                "fallback": bool(r.fallback), "fallback_iterations": r.fallback_iterations,
                "fallback_residual": r.fallback_residual}

    def residual_history(self, cap=4096) -> np.ndarray:
        buf = np.zeros(cap)
        n = ctypes.c_int()
        _check(load().atm_get_residual_history(self.handle, ctypes.c_void_p(buf.ctypes.data), cap, ctypes.byref(n)))
        return buf[: n.value].copy()

    def solution(self, t0=0, count=None, out=None):
        """States t0..t0+count-1 as a float64 tensor on the device (or into `out`,
        a device tensor or host numpy array)."""
        if count is None:
            count = self.level_points(0) - t0
        if out is None:
            out = self.torch.empty((count,) + self.state_shape, dtype=self.torch.float64, device=self.device)
        self._enter()
        _check(load().atm_get_solution(self.handle, t0, count, ctypes.c_void_p(_ptr(out))))
        self._leave()
        return out

    def apply_propagator(self, level, x):
        x = x.to(device=self.device, dtype=self.torch.float64).contiguous()
        out = self.torch.empty_like(x)
        self._enter()
        _check(load().atm_apply_propagator(self.handle, level, ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), x.shape[0]))
        self._leave()
        return out

    def run_stage(self, stage, level=0):
        self._enter()
        _check(load().atm_run_stage(self.handle, stage, level))
        self._leave()

    def level_read(self, level, array, t0=0, count=None):
        if count is None:
            count = self.level_points(level) - t0
        out = self.torch.empty((count,) + self.state_shape, dtype=self.torch.float64, device=self.device)
        self._enter()
        _check(load().atm_level_read(self.handle, level, array, t0, count, ctypes.c_void_p(out.data_ptr())))
        self._leave()
        return out

    def level_write(self, level, array, x, t0=0):
        x = x.to(device=self.device, dtype=self.torch.float64).contiguous()
        self._enter()
        _check(load().atm_level_write(self.handle, level, array, t0, x.shape[0], ctypes.c_void_p(x.data_ptr())))
        self._leave()

    def kernel_profile(self, which):
        """(total ms, launches) of the timed level-0 row (0) or column (1) sweeps."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check(load().atm_get_kernel_profile(self.handle, which, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def sweep_config(self, level=0):
        """Kernels of a level's propagator: dict(kernel, ctas, threads, rows, chunk)."""
        cfg = (ctypes.c_int * 5)()
        _check(load().atm_get_sweep_config(self.handle, level, cfg))
        names = {0: "split", 1: "fused", 2: "learned", 3: "line1d", 4: "chain", 5: "newton", 6: "persistent",
                 7: "float-float"}
        return dict(kernel=names.get(cfg[0], str(cfg[0])), ctas=cfg[1], threads=cfg[2], rows=cfg[3], chunk=cfg[4])

    def newton_stats(self):
        """Gray-Scott counters summed since creation: Newton and GMRES iterations,
        failures, steps, orthogonalisations (basis), line-search trials, GMRES cycles."""
        out = (ctypes.c_longlong * 8)()
        _check(load().atm_get_newton_stats(self.handle, out))
        return dict(newton=out[0], gmres=out[1], failures=out[2], steps=out[3], basis=out[4],
                    trials=out[5], cycles=out[6])

    def set_learned_coarse(self, params):
        """Network weights (torch float32 device tensor) for coarse_prop = PROP_LEARNED or
        PROP_LEARNED_CORRECTION."""
        params = params.to(device=self.device, dtype=self.torch.float32).contiguous()
        self._enter()
        _check(load().atm_set_learned_coarse(self.handle, ctypes.c_void_p(params.data_ptr())))
        self._leave()
        self._nn_params = params

    def level_points(self, level) -> int:
        return load().atm_level_points(self.handle, level)


def batch_solve(solvers, allow_not_converged=True):
    """Solve several Solver objects with one graph launch (atm_batch_solve).
    Returns one result dict per solver."""
    import torch
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    outs = (Result * n)()
    cur = torch.cuda.current_stream(solvers[0].device)
    for s in solvers:
        cur.wait_stream(s.stream)
    st = load().atm_batch_solve(hs, n, ctypes.c_void_p(cur.cuda_stream), outs)
    _check(st, (0, 4) if allow_not_converged else (0,))
    res = []
    for s, r in zip(solvers, outs):
        s.stream.wait_stream(cur)
        res.append({"iterations": r.iterations, "converged": bool(r.converged),
                    "initial_residual": r.initial_residual, "final_residual": r.final_residual,
                    "time_ms": r.time_ms})
    return res


class LearnedCoarse:
    """The learned coarse propagator Psi_NN(u) = u + N(u) (include/atm.h):
    inference, loss/gradient and Adam training through the C ABI, on torch
    float32 device tensors of shape (n, ny, nx)."""

    def __init__(self, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.nparams = load().atm_nn_param_count()
        self._ws = {}

    def _workspace(self, n, ny, nx, training):
        key = (n, ny, nx, training)
        if key not in self._ws:
            b = ctypes.c_size_t()
            _check(load().atm_nn_workspace_size(n, nx, ny, int(training), ctypes.byref(b)))
            self._ws[key] = self.torch.empty(b.value + 256, dtype=self.torch.uint8, device=self.device)
        w = self._ws[key]
        base = (w.data_ptr() + 255) // 256 * 256
        return ctypes.c_void_p(base), w.numel() - 256

    def _sync_in(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _sync_out(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def apply(self, params, u):
        u = u.to(device=self.device, dtype=self.torch.float32).contiguous()
        out = self.torch.empty_like(u)
        n, ny, nx = u.shape
        ws, nb = self._workspace(n, ny, nx, False)
        self._sync_in()
        _check(load().atm_nn_apply(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), n, nx, ny, ws, nb,
                                   ctypes.c_void_p(self.stream.cuda_stream)))
        self._sync_out()
        return out

    def loss_grad(self, params, u, target):
        u = u.to(device=self.device, dtype=self.torch.float32).contiguous()
        target = target.to(device=self.device, dtype=self.torch.float32).contiguous()
        n, ny, nx = u.shape
        grad = self.torch.empty(self.nparams, dtype=self.torch.float32, device=self.device)
        loss = ctypes.c_double()
        ws, nb = self._workspace(n, ny, nx, True)
        self._sync_in()
        _check(load().atm_nn_loss_grad(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                       ctypes.c_void_p(target.data_ptr()), n, nx, ny,
                                       ctypes.c_void_p(grad.data_ptr()), ctypes.byref(loss), ws, nb,
                                       ctypes.c_void_p(self.stream.cuda_stream)))
        self._sync_out()
        return loss.value, grad

    def train(self, params, adam, inputs, targets, steps, batch, lr=1e-3, beta1=0.9, beta2=0.999,
              eps=1e-8, log_every=50):
        """Adam steps on (inputs, targets) pairs; params and adam (2 * nparams zeros
        at the start) are updated in place.  Returns (losses, result dict)."""
        n, ny, nx = inputs.shape
        hist = np.zeros(steps // max(log_every, 1) + 2, dtype=np.float32)
        cfg = TrainCfg(steps, batch, lr, beta1, beta2, eps, log_every,
                       ctypes.c_void_p(hist.ctypes.data), hist.size)
        res = TrainResult()
        ws, nb = self._workspace(batch, ny, nx, True)
        self._sync_in()
        _check(load().atm_train_learned_coarse(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(adam.data_ptr()),
                                               ctypes.c_void_p(inputs.data_ptr()), ctypes.c_void_p(targets.data_ptr()),
                                               n, nx, ny, ctypes.byref(cfg), ctypes.byref(res), ws, nb,
                                               ctypes.c_void_p(self.stream.cuda_stream)))
        self._sync_out()
        return hist[: res.logged].copy(), {"steps": res.steps, "final_loss": res.final_loss,
                                            "time_ms": res.time_ms}
