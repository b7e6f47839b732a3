"""Benchmark: AT-MGRIT time-to-solution on one GB300 (or N, one independent
problem per rank), printed as one JSON line.

Workload (default): 2D Allen-Cahn, 256^2 periodic grid, eps = 0.02, PR-ADI
fine step with explicit reaction, 4097 time points, dt = 1e-4, three-level
AT-MGRIT, m = (16, 16), local grids of k = 8 points, FCF relaxation, residual
tolerance 1e-8, u0 ~ U(-0.05, 0.05) (seed = rank), zero initial guess.
A step is one full solve to ||r||_2 <= 1e-8 from the zero guess: every row of
the sweep (relaxation, residual, restriction, local chains, correction, norm,
cycle control).  value = fine time steps resolved per second
= ranks * (nt - 1) / time-to-solution.  Default arithmetic: FP32 propagation
inside the FP64 refinement loop (FP64 iterate, residual, update and norm),
the residual pass's fine propagator evaluated in float-float (pairs of FP32,
~48-bit significands, on the FP32 pipes); the line states the error of the
result against the oracle's FP64 sequential solution.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl atm|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import atm_inputs as I  # noqa: E402

METRIC = "time-to-solution at residual 1e-8 and fine steps/s; HBM GB/s vs peak; AT-MGRIT vs plain"
UNIT = "fine steps/s"

WORKLOADS = {
    "allen_cahn_256": dict(kind="ac", n=256, nt=4097, dt=1e-4, eps=0.02, m=(16, 16), k=8, nu=1,
                           tol=1e-8, max_iter=60),
    "heat1d_127": dict(kind="heat1d", n=127, nt=1025, dt=1 / 1024, eps=0.0, m=(8,), k=4, nu=1,
                       tol=1e-10, max_iter=60),
    # 1024^2 x 65537 with m = (32, 4, 4), k = 16: FP32 with C-point storage (the FP64
    # kernels stop at 512); tol = RMS 2e-7 per C-point value, near the FP32 floor
    "allen_cahn_1024": dict(kind="ac", n=1024, nt=65537, dt=2.5e-5, eps=0.02, m=(32, 4, 4), k=16, nu=1,
                            tol=1e-2, max_iter=30),
}

# Arithmetic forms (--precision): FP64; FP32; FP32 propagation inside the FP64
# refinement loop; the same with the FP64 residual pass's fine propagator in
# float-float (pairs of FP32, ~48-bit significands); FP64 with that fine
# propagator.
PRECISIONS = {"fp64": lambda a: a.FP64, "fp32": lambda a: a.FP32, "fp32r": lambda a: a.FP32_REFINED,
              "fp32rf": lambda a: a.FP32_REFINED_FF, "fp64f": lambda a: a.FP64_FF}

# Textbook flops per grid value of one sweep kernel:
# PR explicit term 5, periodic tridiagonal solve 7 (Thomas 5 + rank-one
# periodic correction 2), split-BE right-hand side 0, reaction substep 5,
# Dirichlet tridiagonal solve 5 (+2 for the first-row correction).
FLOPS_PER_VALUE = {("row", "pr_react"): 17, ("row", "pr"): 12, ("col", "pr"): 12,
                   ("row", "split"): 7, ("col", "split"): 7, ("row", "heat1d"): 7}


def load_json(path, default=None):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return default


# FP64 rate derived from unit counts and clocks: 152 SMs x 2 FP64 FMA per
# clock x 2 flop x 2.07 GHz (GB300's FP64 rate, 1/64 of FP32)
FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def peaks(fp64_measured=None):
    mp = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"), {}) or {}
    return {
        "hbm_gbs": mp.get("hbm_gbs", 6800.0),
        "hbm_src": "measured" if "hbm_gbs" in mp else "fallback",
        "fp64_tflops": fp64_measured if fp64_measured else FP64_DERIVED_TFLOPS,
        "fp64_src": (f"measured FP64 FMA probe on this GPU (atm_measure_fp64_rate; derived peak "
                     f"{FP64_DERIVED_TFLOPS:.3f})" if fp64_measured else
                     "derived FP64 FMA rate (152 SMs x 2 FMA/clk x 2.07 GHz)"),
    }


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(kind="split"):
    """Hash of the timed kernel's source (the split sweep kernels, the fused
    cluster kernels or the float-float kernel): stored ncu traffic is used only
    while it matches."""
    name = {"fused": "atm_fused.cuh", "persistent": "atm_fused.cuh", "float-float": "atm_df.cuh"}.get(kind,
                                                                                                 "atm_kernels.cuh")
    with open(os.path.join(ROOT, "paper_2107_09596_gb300", "csrc", name), "rb") as fh:
        return hashlib.md5(fh.read()).hexdigest()[:12]


def batch_descs(atm, count=64, seed=0, precision="fp32r", storage="cpoint"):
    """The batched workload: `count` problems drawn by atm_inputs.batch_problem_draws
    (kind in {heat2d, Allen-Cahn}, n in {64..512}, nt in {1025, 4097, 16385},
    m in {8, 16}); AT-MGRIT FCF with two coarsenings when the coarse grid allows,
    k = ceil(N_c / 4); dt = 1e-4, eps = 0.02.  fp32r / fp32rf (FP32 propagation,
    FP64 residual in FP64 or float-float) and fp64: stop at an RMS C-point
    residual of 1e-10 per value; fp32: at an RMS residual of 1e-6 (the FP32 floor
    is near 1e-7)."""
    out = []
    for d in I.batch_problem_draws(count, seed):
        kind = atm.ALLEN_CAHN if d["kind"] == "allen_cahn" else atm.HEAT2D
        n, nt, m = d["n"], d["nt"], d["m"]
        prob = atm.make_problem(kind, n, n, dt=1e-4, nt_points=nt, eps=0.02)
        nc = (nt - 1) // m + 1
        ms = (m, m) if (nc - 1) // m + 1 >= 3 else (m,)
        nco = ((nc - 1) // m + 1) if len(ms) == 2 else nc
        k = max(2, (nco + 3) // 4)
        rms = 1e-6 if precision == "fp32" else 1e-10
        pts = nc if storage == "cpoint" else nt
        prec = {"fp32r": atm.FP32_REFINED, "fp32rf": atm.FP32_REFINED_FF, "fp64": atm.FP64,
                "fp32": atm.FP32}[precision]
        desc = atm.make_solver(atm.AT_MGRIT, m=ms, k=k, nu=1, tol=rms * np.sqrt(pts * n * n),
                               max_iter=40, precision=prec, use_graph=2, cpoint_only=storage == "cpoint")
        out.append((d, prob, desc))
    return out


def run_batch(args):
    """One graph launch per memory group (atm_batch_solve) against the same
    problems solved one at a time (each one device-side loop launch)."""
    import torch
    import paper_2107_09596_gb300 as atm
    device = torch.device("cuda", 0)
    atm._build.build()
    bprec = args.precision if args.precision in ("fp32r", "fp32rf", "fp32") else "fp32rf"
    descs = batch_descs(atm, precision=bprec, storage=args.storage)
    budget = 240e9
    groups, cur, used = [], [], 0
    for item in descs:
        b = atm.workspace_size(item[1], item[2])
        if cur and used + b > budget:
            groups.append(cur)
            cur, used = [], 0
        cur.append(item)
        used += b
    groups.append(cur)
    total_steps = sum(d["nt"] - 1 for d, _, _ in descs)
    t_batch = t_single = 0.0
    iters_b, iters_s, statuses, failed, ms_single = [], [], [], [], []
    for g in groups:
        solvers = [atm.Solver(p, s, device=device) for _, p, s in g]
        for (d, _, _), sv in zip(g, solvers):
            sv.set_initial_condition(torch.as_tensor(I.uniform_field((d["n"], d["n"]), d["seed"]),
                                                     dtype=torch.float64, device=device))
        torch.cuda.synchronize()
        # one at a time (device-side loop per solve), then the batch from the same state
        t = time.perf_counter()
        for sv in solvers:
            sv.set_initial_guess(None)
            t1 = time.perf_counter()
            r = sv.solve()
            ms_single.append((time.perf_counter() - t1) * 1e3)
            iters_s.append(r["iterations"])
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t
        for sv in solvers:
            sv.set_initial_guess(None)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = atm.batch_solve(solvers)
        torch.cuda.synchronize()
        t_batch += time.perf_counter() - t
        iters_b += [r["iterations"] for r in res]
        statuses += [r["converged"] for r in res]
        for (d, p, s), sv, r in zip(g, solvers, res):
            if not r["converged"]:
                h = sv.residual_history()
                failed.append({"draw": descs.index((d, p, s)), "kind": d["kind"], "n": d["n"], "nt": d["nt"],
                               "m": list(s.m[:s.levels - 1]),
                               "k": s.k, "cycles": r["iterations"], "tol": s.tol,
                               "residual_history": [float(x) for x in h[:8]] + ([float(h[-1])] if len(h) > 8 else [])})
        for sv in solvers:
            sv.close()
        del solvers
        torch.cuda.empty_cache()
    # the plain FP64 form of the same problems to the same tolerances, one at a time
    t_fp64, conv64 = None, None
    if args.batch_fp64:
        t_fp64, conv64 = 0.0, 0
        for d, p, s in batch_descs(atm, precision="fp64", storage=args.storage):
            sv = atm.Solver(p, s, device=device)
            sv.set_initial_condition(torch.as_tensor(I.uniform_field((d["n"], d["n"]), d["seed"]),
                                                     dtype=torch.float64, device=device))
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = sv.solve()
            torch.cuda.synchronize()
            t_fp64 += time.perf_counter() - t
            conv64 += int(r["converged"])
            sv.close()
            torch.cuda.empty_cache()
    value = total_steps / t_batch
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32r": "f32+f64", "fp32rf": "f32+f32x2", "fp32": "f32"}[bprec], "data": "synthetic",
            "config": {"workload": "batch64", "problems": len(descs), "groups": len(groups),
                       "precision": bprec, "storage": args.storage,
                       "memory_budget_gb_per_group": budget / 1e9, "l2": "inputs larger than L2"},
            "one_at_a_time": {"value": total_steps / t_single, "ms": t_single * 1e3,
                              "ms_per_problem": [round(x, 2) for x in ms_single]},
            "batched_speedup": t_single / t_batch,
            "iterations_batched": iters_b, "iterations_one_at_a_time": iters_s,
            "converged": int(sum(statuses)), "not_converged": failed,
            "plain_fp64_one_at_a_time": None if t_fp64 is None else {
                "ms": t_fp64 * 1e3, "value": total_steps / t_fp64, "converged": conv64}}
    print(json.dumps(line), flush=True)


# Gray-Scott of Sec. 5.1: 128^2 on the periodic [0, 2.5]^2, 16384 points on
# [0, 256], backward Euler with Newton (tolerance 1e-10), stop at the space-time
# residual 1e-7, nested iteration; the paper's two-level (m = 64, k = 128,
# F-relaxation; Table 1) and three-level ((64, 4), k = 32, FCF; Table 2) forms.
GS_WORKLOAD = dict(n=128, nt=16384, dt=256.0 / 16383.0, lx=2.5, tol=1e-7, max_iter=30,
                   newton_tol=1e-10, du=8e-5, dv=4e-5, feed=0.024, kill=0.06)
GS_CONFIGS = {"2lvl": dict(m=(64,), k=128, nu=0), "3lvl": dict(m=(64, 4), k=32, nu=1)}
# the other rows of Tables 1 and 2 (k = half the coarsest grid's points)
GS_CONFIGS.update({f"2lvl_m{mm}": dict(m=(mm,), k=8192 // mm, nu=0) for mm in (128, 256, 512)})
GS_CONFIGS.update({f"3lvl_64_{m1}": dict(m=(64, m1), k=128 // m1, nu=1) for m1 in (2, 8, 16)})
GS_METRIC = "Gray-Scott time-to-solution at space-time residual 1e-7 and fine steps/s"


def gs_vector_bytes(st, n2):
    """Bytes of whole-vector reads and writes (2 n^2 values) done by the Newton
    kernel as written, from its counters.  FP64 passes: per step 7, per Newton
    iteration -4 (including the read of the iterate for its FP32 copy), per
    line-search trial 6, per GMRES cycle 9.  FP32 passes (Krylov basis,
    preconditioner, the iterate's FP32 copy): per Newton iteration 1, per GMRES
    cycle 18, per GMRES iteration 22, per basis vector orthogonalised against 4."""
    f64 = 7 * st["steps"] - 4 * st["newton"] + 6 * st["trials"] + 9 * st["cycles"]
    f32 = st["newton"] + 18 * st["cycles"] + 22 * st["gmres"] + 4 * st["basis"]
    return (8 * f64 + 4 * f32) * n2


def run_gs_probe(args):
    """One level-0 and one level-1 Newton launch of the two-level Gray-Scott
    handle on 255 states (0.7 x the initial state + 0.3 x seeded random
    states): the small case for profiling the Newton kernel."""
    import torch
    import paper_2107_09596_gb300 as atm
    w = dict(GS_WORKLOAD, **GS_CONFIGS["2lvl"])
    atm._build.build()
    n = w["n"]
    prob = atm.make_problem(atm.GRAY_SCOTT, n, n, lx=w["lx"], ly=w["lx"], dt=w["dt"], nt_points=w["nt"],
                            du=w["du"], dv=w["dv"], feed=w["feed"], kill=w["kill"],
                            newton_tol=w["newton_tol"], newton_max_iter=50)
    desc = atm.make_solver(atm.AT_MGRIT, m=w["m"], k=w["k"], nu=w["nu"], tol=w["tol"], max_iter=w["max_iter"],
                           cpoint_only=True)
    s = atm.Solver(prob, desc)
    x = np.stack([0.3 * I.gray_scott_random_state(n, n, seed) + 0.7 * I.gray_scott_initial_condition(n, n)
                  for seed in range(255)])
    xd = torch.as_tensor(x, device="cuda:0")
    ms = []
    for level in (0, 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.apply_propagator(level, xd)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"gs_probe": {"states": 255, "level_ms": ms, "newton": s.newton_stats()}}))
    s.close()


def run_gray_scott(args):
    import torch
    import paper_2107_09596_gb300 as atm
    w = dict(GS_WORKLOAD, **GS_CONFIGS[args.gs_config])
    if args.max_iter is not None:
        w["max_iter"] = args.max_iter
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    atm._build.build()
    n = w["n"]
    prob = atm.make_problem(atm.GRAY_SCOTT, n, n, lx=w["lx"], ly=w["lx"], dt=w["dt"], nt_points=w["nt"],
                            du=w["du"], dv=w["dv"], feed=w["feed"], kill=w["kill"],
                            newton_tol=w["newton_tol"], newton_max_iter=50)
    alg = {"at": atm.AT_MGRIT, "mgrit": atm.MGRIT, "seq": atm.SEQUENTIAL}[args.algorithm]
    nested = not args.cold and args.algorithm != "seq"
    desc = atm.make_solver(alg, m=w["m"], k=w["k"], nu=w["nu"], tol=w["tol"], max_iter=w["max_iter"],
                           precision=atm.FP64, use_graph=2 if args.algorithm != "seq" else True,
                           cpoint_only=args.storage == "cpoint", nested=nested)
    solver = atm.Solver(prob, desc, device=device)
    u0 = torch.as_tensor(I.gray_scott_initial_condition(n, n), dtype=torch.float64, device=device)

    def step():
        solver.set_initial_guess(None)
        solver.set_initial_condition(u0)
        return solver.solve()

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize(device)
    st0 = solver.newton_stats()
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches, iters = 0, []
    e0.record(solver.stream)
    for _ in range(args.steps):
        res = step()
        launches += res["launches"]
        iters.append(res["iterations"])
    e1.record(solver.stream)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st1 = solver.newton_stats()
    d = {k: (st1[k] - st0[k]) / args.steps for k in st1}
    value = (w["nt"] - 1) / (ms / 1e3)
    hist = solver.residual_history()

    # end to end: the initial state from pinned host memory, the final state and
    # the residual history back, inside the timed region
    shape = solver.state_shape
    h_u0 = torch.as_tensor(I.gray_scott_initial_condition(n, n), dtype=torch.float64).pin_memory()
    h_out = torch.empty(shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(device)
    t = time.perf_counter()
    for _ in range(args.steps):
        solver.set_initial_guess(None)
        solver.set_initial_condition(h_u0)
        solver.solve()
        solver.solution(w["nt"] - 1, 1, out=h_out)
        h2 = solver.residual_history()
    torch.cuda.synchronize(device)
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps
    state_bytes = int(np.prod(shape)) * 8

    # roofline of the Newton kernel: whole-vector passes (from its counters)
    # over the timed region, against the measured HBM copy rate
    pk = peaks()
    nbytes = gs_vector_bytes(d, int(np.prod(shape)))
    achieved = nbytes / (ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": None,
            "kernel": "gs_newton_kernel (every propagator application of the solve)",
            "peak_source": f"{pk['hbm_src']} STREAM copy (MEASURED_PEAKS.json)",
            "algorithmic": f"{nbytes / 1e9:.1f} GB of whole-vector passes per solve (Newton kernel as "
                           f"written: counters x passes per event, FP64 and FP32 vectors) / timed solve "
                           f"time (includes the few non-Newton kernels: a lower bound of the kernel's "
                           f"own rate)"}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        c = oracle.make_cfg(oracle.GRAY_SCOTT, n, n, lx=w["lx"], ly=w["lx"], dt=w["dt"], nt=3, m=(2,),
                            gs=dict(du=w["du"], dv=w["dv"], feed=w["feed"], kill=w["kill"],
                                    tol=w["newton_tol"], max_iter=50))
        x = I.gray_scott_initial_condition(n, n)[None]
        steps_cpu = 6
        t = time.perf_counter()
        for _ in range(steps_cpu):
            x = oracle.apply_prop(c, 0, x)
        sec = time.perf_counter() - t
        cpu = {"value": steps_cpu / sec, "unit": "fine steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{steps_cpu} sequential backward Euler Newton steps of the oracle from the "
                         f"initial state ({sec:.1f} s; sparse LU per Newton iteration): its sequential "
                         f"stepping rate, the fastest the oracle covers the time axis"}
    line = {"metric": GS_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic (the paper's initial state)",
            "config": {"workload": "gray_scott_128", "gs_config": args.gs_config,
                       **{k: (list(v) if isinstance(v, tuple) else v) for k, v in w.items()},
                       "algorithm": args.algorithm, "storage": args.storage, "nested": nested,
                       "l2": "working set larger than L2 (Newton scratch %.2f GB)" % (
                           atm.workspace_size(prob, desc) / 1e9)},
            "iterations": int(np.median(iters)), "time_to_solution_ms": ms,
            "final_residual": float(res["final_residual"]),
            "residual_history": [float(v) for v in hist][:64],
            "newton_per_solve": d,
            "e2e": {"value": (w["nt"] - 1) / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes + 8 * len(h2)},
            "gpu_launches": int(launches),
            "kernels_per_level": [solver.sweep_config(0)],
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line), flush=True)
    solver.close()


def run_nn_probe(args):
    """Inference of the learned coarse propagator alone (the tensor-core
    convolutions of Psi_NN, five layers) on 32 states of the workload's grid,
    timed with CUDA events on the network's stream, against the measured bf16
    tensor peak.  Algorithmic work per pixel: 2 * 9 * (1*32 + 3*32*32 + 32*1)
    = 56,448 flop (the kernels pad the first layer's K and the last layer's N
    to 16, which is not counted)."""
    import torch
    import paper_2107_09596_gb300 as atm
    atm._build.build()
    w = WORKLOADS[args.workload]
    n, states = w["n"], 32
    net = atm.LearnedCoarse()
    flat = np.concatenate([np.concatenate([wt.ravel(), b.ravel()]) for (wt, b) in I.conv_net_init(7)])
    params = torch.as_tensor(flat, dtype=torch.float32, device="cuda:0")
    x = torch.as_tensor(I.uniform_field((states, n, n), 1, -1.0, 1.0), dtype=torch.float32, device="cuda:0")
    for _ in range(max(args.warmup, 1)):
        net.apply(params, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 1)
    e0.record(net.stream)
    for _ in range(reps):
        net.apply(params, x)
    e1.record(net.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flop = 2 * 9 * (1 * 32 + 3 * 32 * 32 + 32 * 1) * n * n * states
    mp = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"), {}) or {}
    peak = mp.get("bf16_tflops", 1900.0)
    ach = flop / (ms / 1e3) / 1e12
    print(json.dumps({"probe": "learned coarse propagator inference (five tcgen05 convolution layers)",
                      "states": states, "grid": [n, n], "ms_per_apply": ms,
                      "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                   "frac": ach / peak,
                                   "peak_source": ("measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"
                                                   if "bf16_tflops" in mp else "fallback"),
                                   "algorithmic": "56,448 flop per pixel (five 3x3 layers, 1-32-32-32-32-1)"}}),
          flush=True)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "atm" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def train_learned(atm, w, device, steps, seeds=tuple(range(101, 117)), cycles=(1, 2, 3, 5, 8), batch=8,
                  correction=False):
    """Psi_NN for the workload's level-1 step (m_0 fine steps), trained by Adam
    on the pairs (u_C, Phi^m0 u_C) that the method's own F-relaxation generates
    in the first cycles of FP32 AT-MGRIT solves of other seeds
    (training.method_pairs: after c cycles, the C-points of the iterate and
    their F-relaxation).  correction: train the network on
    Phi^m0(u) - Psi_split(u) + u, for the corrected propagator Psi_split(u) + N(u)."""
    import torch
    from paper_2107_09596_gb300.training import method_pairs
    prob, _ = make_desc(atm, w, "at", atm.FP32, profile=False)

    def desc(c):
        _, d = make_desc(atm, w, "at", atm.FP32, profile=False)
        d.tol, d.max_iter = 0.0, c
        return d

    u0s = [torch.as_tensor(initial_condition(w, sd), dtype=torch.float64, device=device) for sd in seeds]
    inputs, targets = method_pairs(prob, desc, u0s, cycles, device=device)
    if correction:
        prob, d64 = make_desc(atm, w, "at", atm.FP64, profile=False)
        cl = atm.Solver(prob, d64, device=device)
        for i in range(0, inputs.shape[0], 64):
            x = inputs[i:i + 64].to(torch.float64)
            targets[i:i + 64] -= (cl.apply_propagator(1, x) - x).to(torch.float32)
        cl.close()
    net = atm.LearnedCoarse(device=device)
    flat = np.concatenate([np.concatenate([wt.ravel(), b.ravel()]) for (wt, b) in I.conv_net_init(7)])
    params = torch.as_tensor(flat, dtype=torch.float32, device=device)
    adam = torch.zeros(2 * net.nparams, dtype=torch.float32, device=device)
    perm = torch.randperm(inputs.shape[0], generator=torch.Generator().manual_seed(0)).to(device)
    inputs, targets = inputs[perm].contiguous(), targets[perm].contiguous()
    hist, res = net.train(params, adam, inputs, targets, steps=steps, batch=batch, lr=1e-3, log_every=250)
    return params, {"pairs": int(inputs.shape[0]), "data": f"method F-relaxation pairs: seeds {seeds[0]}-"
                    f"{seeds[-1]}, iterates after {list(cycles)} FP32 AT-MGRIT cycles", "steps": steps,
                    "batch": batch, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                    "train_ms": res["time_ms"]}


def make_desc(atm, w, algorithm, precision, profile, coarse="classical", sweep="auto", cpoint=False,
              inner_cycles=0, nu=None, nested=False, fcycle=False, inner_coarse_relax=0):
    kind = {"ac": atm.ALLEN_CAHN, "heat1d": atm.HEAT1D}[w["kind"]]
    ny = w["n"] if w["kind"] != "heat1d" else 1
    prob = atm.make_problem(kind, w["n"], ny, dt=w["dt"], nt_points=w["nt"], eps=w["eps"])
    alg = {"at": atm.AT_MGRIT, "mgrit": atm.MGRIT, "seq": atm.SEQUENTIAL}[algorithm]
    desc = atm.make_solver(alg, m=w["m"], k=w["k"], nu=w["nu"] if nu is None else nu, tol=w["tol"],
                           max_iter=w["max_iter"], precision=precision, use_graph=True,
                           profile=profile,
                           coarse_prop={"learned": atm.PROP_LEARNED, "correction": atm.PROP_LEARNED_CORRECTION}.get(
                               coarse, atm.PROP_SPLIT_BE),
                           sweep_kernel={"auto": atm.SWEEP_AUTO, "split": atm.SWEEP_SPLIT,
                                         "fused": atm.SWEEP_FUSED, "chain": atm.SWEEP_CHAIN,
                                         "persistent": atm.SWEEP_PERSISTENT}[sweep],
                           cpoint_only=cpoint, inner_cycles=inner_cycles, nested=nested, fcycle=fcycle,
                           inner_coarse_relax=inner_coarse_relax)
    return prob, desc


def initial_condition(w, seed):
    if w["kind"] == "heat1d":
        return I.heat1d_initial_condition(w["n"], seed)
    return I.uniform_field((w["n"], w["n"]), seed)


def oracle_cfg(w):
    import oracle
    kind = {"ac": oracle.ALLEN_CAHN, "heat1d": oracle.HEAT1D}[w["kind"]]
    ny = w["n"] if w["kind"] != "heat1d" else 1
    return oracle.make_cfg(kind, w["n"], ny, dt=w["dt"], nt=w["nt"], eps=w["eps"], m=w["m"],
                           k=w["k"], nu=w["nu"], react_exact=[l > 0 for l in range(len(w["m"]) + 1)])


def oracle_sequential_baseline(w, seed):
    """CPU baseline: the oracle (as it stands) solves the same workload
    completely by sequential time stepping -- the fixed point every solver
    converges to (Sec. 2), exact up to rounding -- on one host core.  Returns
    the baseline entry and the oracle's C-points (every m_0-th state), from
    which the GPU result's error is stated."""
    import oracle
    c = oracle_cfg(w)
    u0 = initial_condition(w, seed)
    t = time.perf_counter()
    u = oracle.sequential(c, u0)
    sec = time.perf_counter() - t
    cps = u[::w["m"][0]].copy()
    del u
    return {"value": (w["nt"] - 1) / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one complete solve of this workload by the oracle's sequential time stepping "
                      f"(FP64, {w['nt'] - 1} steps, {sec:.1f} s, measured; the oracle's AT-MGRIT solve "
                      f"on all cores is the --impl reference line)"}, cps


def error_vs_oracle(solver, w, cps):
    """Relative L2 error of the GPU iterate against the oracle's sequential
    solution: every C-point (state by state and over all of them) and the
    final state."""
    m0 = w["m"][0]
    got = np.stack([solver.solution(t, 1).cpu().numpy()[0] for t in range(0, w["nt"], m0)])
    per = [float(np.linalg.norm(got[i] - cps[i]) / max(np.linalg.norm(cps[i]), 1e-300))
           for i in range(1, got.shape[0])]
    tot = float(np.linalg.norm(got[1:] - cps[1:]) / np.linalg.norm(cps[1:]))
    fin = solver.solution(w["nt"] - 1, 1).cpu().numpy()[0]
    ref_fin = cps[-1] if (w["nt"] - 1) % m0 == 0 else None
    out = {"against": "oracle sequential solution (FP64, same initial condition)",
           "rel_l2_cpoints": tot, "max_rel_l2_per_cpoint": max(per), "cpoints": len(per)}
    if ref_fin is not None:
        out["rel_l2_final_state"] = float(np.linalg.norm(fin - ref_fin) / np.linalg.norm(ref_fin))
    return out


def run_reference(args, w, world, rank, dist, budget_s=150.0):
    """--impl reference: the oracle's AT-MGRIT (FP64, all host cores, the same
    workload, cycle and tolerance) on rank 0 only.  Each timed step is one
    complete solve from the zero guess to ||r||_2 <= tol; a solve takes tens of
    seconds, so the run times as many solves as fit in budget_s (at least one)
    and reports that count in `steps`.  Warm-up: one V-cycle (untimed)."""
    if rank != 0:
        return
    import oracle
    c = oracle_cfg(w)
    u0 = initial_condition(w, 0)
    u = np.zeros((w["nt"],) + oracle.state_shape(c))
    u[0] = u0
    oracle.solve(c, u, 1, 0.0)          # warm-up: pages the iterate in, one cycle
    times, iters, finals = [], [], []
    t_start = time.perf_counter()
    while not times or (len(times) < args.steps and
                        time.perf_counter() - t_start + float(np.mean(times)) <= budget_s):
        u[1:] = 0.0
        u[0] = u0
        t = time.perf_counter()
        it, hist = oracle.solve(c, u, w["max_iter"], w["tol"])
        times.append(time.perf_counter() - t)
        iters.append(int(it))
        finals.append(float(hist[-1]))
    sec = float(np.mean(times))
    value = (w["nt"] - 1) / sec
    sample = (f"{len(times)} complete AT-MGRIT solves of the oracle (FP64, {oracle.num_threads()} threads, "
              f"zero guess to ||r||_2 <= {w['tol']:g}: {iters[0]} cycles, final residual {finals[0]:.2e}), "
              f"measured; warm-up: one V-cycle")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": 1, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, **{k: (list(v) if isinstance(v, tuple) else v)
                                                     for k, v in w.items()},
                       "algorithm": "at", "l2": "inputs larger than L2 (host run)"},
            "iterations": iters[0], "final_residual": finals[0],
            "steps_requested": args.steps, "solve_times_s": times,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["atm", "reference"], default="atm")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch64", "gray_scott_128"],
                    default="allen_cahn_256",
                    help="batch64: 64 drawn problems, batched against one at a time; gray_scott_128: the "
                         "Gray-Scott problem of Sec. 5.1 (neither is the default)")
    ap.add_argument("--gs-config", choices=sorted(GS_CONFIGS), default="2lvl",
                    help="gray_scott_128: 2lvl (m = 64, k = 128, F), 3lvl ((64, 4), k = 32, FCF), or "
                         "another row of Tables 1-2: 2lvl_m128/256/512, 3lvl_64_2/8/16")
    ap.add_argument("--cold", action="store_true", help="gray_scott_128: zero guess instead of nested iteration")
    ap.add_argument("--gs-probe", action="store_true",
                    help="gray_scott_128: only one level-0 and one level-1 Newton launch on 255 states "
                         "(the profiling case)")
    ap.add_argument("--algorithm", choices=["at", "mgrit", "seq"], default="at")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32rf",
                    help="fp32r: FP32 propagation with FP64 refinement; fp32rf: the same with the FP64 residual "
                         "pass in float-float (pairs of FP32); fp64f: FP64 with the fine propagator in float-float")
    ap.add_argument("--coarse", choices=["classical", "learned", "correction"], default="classical",
                    help="level-1 coarse propagator; 'learned' trains Psi_NN, 'correction' the network of "
                         "Psi_split + N first (untimed)")
    ap.add_argument("--train-steps", type=int, default=2500)
    ap.add_argument("--sweep-kernel", choices=["auto", "split", "fused", "chain", "persistent"], default="auto",
                    help="2D propagator kernels (auto: level 0 autotuned at create time)")
    ap.add_argument("--storage", choices=["cpoint", "full"], default="cpoint",
                    help="level-0 storage: C-points only (default) or every time point")
    ap.add_argument("--nu", type=int, choices=[0, 1], default=None,
                    help="relaxation: 0 F, 1 FCF (default: the workload's); in fp32r it shapes the inner cycles")
    ap.add_argument("--inner-coarse-relax", choices=["F", "nu"], default="F",
                    help="refined modes: relaxation on the coarse levels of the FP32 inner cycles (F, or as --nu)")
    ap.add_argument("--inner-cycles", type=int, default=0,
                    help="fp32r: FP32 V-cycles per FP64 refinement step (0: the library default, 5)")
    ap.add_argument("--max-iter", type=int, default=None, help="override the workload's cycle cap")
    ap.add_argument("--nested", action="store_true", help="nested iteration: start from the coarse hierarchy")
    ap.add_argument("--fcycle", action="store_true", help="F-cycles instead of V-cycles")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-fp64", action="store_true",
                    help="batch64: also solve the problems in plain FP64, one at a time, to the same tolerances")
    ap.add_argument("--nn-probe", action="store_true",
                    help="time the learned propagator's tensor-core inference alone (32 states of the workload's "
                         "grid) and print its roofline")
    ap.add_argument("--tune-cache-out", default=None,
                    help="write the autotuner's kernel choices of this run to this file")
    ap.add_argument("--tune-cache-in", default=None,
                    help="use the kernel choices recorded in this file (e.g. a profiler run replaying the kernels "
                         "of a timed run)")
    args = ap.parse_args()
    if args.workload == "batch64":
        run_batch(args)
        return
    if args.workload == "gray_scott_128":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "gray_scott_128 has no reference arm; "
                              "its CPU baseline is the oracle's stepping rate in the atm line"}))
            return
        if args.gs_probe:
            run_gs_probe(args)
        else:
            run_gray_scott(args)
        return
    if args.nn_probe:
        run_nn_probe(args)
        return
    w = dict(WORKLOADS[args.workload])
    if args.max_iter is not None:
        w["max_iter"] = args.max_iter
    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, w, world, rank, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch
    import paper_2107_09596_gb300 as atm
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    atm._build.build()
    prec = PRECISIONS[args.precision](atm)
    if args.tune_cache_in:
        with open(args.tune_cache_in) as fh:
            atm.tune_cache_import(fh.read())
    learned_info = None
    if args.coarse in ("learned", "correction"):
        nn_params, learned_info = train_learned(atm, w, device, args.train_steps,
                                                correction=args.coarse == "correction")
    prob, desc = make_desc(atm, w, args.algorithm, prec, profile=True, coarse=args.coarse,
                           sweep=args.sweep_kernel, cpoint=args.storage == "cpoint",
                           inner_cycles=args.inner_cycles, nu=args.nu, nested=args.nested, fcycle=args.fcycle,
                           inner_coarse_relax=int(args.inner_coarse_relax == "nu"))
    solver = atm.Solver(prob, desc, device=device)
    if args.coarse in ("learned", "correction"):
        solver.set_learned_coarse(nn_params)
    shape = solver.state_shape
    u0 = torch.as_tensor(initial_condition(w, rank), dtype=torch.float64, device=device)

    def step():
        solver.set_initial_guess(None)
        solver.set_initial_condition(u0)
        return solver.solve()

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize(device)
    prof0 = [solver.kernel_profile(i) for i in range(4)]
    clocks = ClockSampler(device.index if device.index is not None else 0)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    iters = []
    fallbacks = []
    e0.record(solver.stream)
    for _ in range(args.steps):
        res = step()
        launches += res["launches"]
        iters.append(res["iterations"])
        fallbacks.append((res["fallback"], res["fallback_iterations"], res["fallback_residual"]))
    e1.record(solver.stream)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    barrier(dist, device)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(dist, ms, device)
    value = world * (w["nt"] - 1) / (ms / 1e3)
    prof1 = [solver.kernel_profile(i) for i in range(4)]

    # end to end through host buffers: u0 from pinned host memory in, the final
    # state and the residual history out, copies inside the timed region
    h_u0 = torch.as_tensor(initial_condition(w, rank), dtype=torch.float64).pin_memory()
    h_out = torch.empty(shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(device)
    barrier(dist, device)
    t = time.perf_counter()
    for _ in range(args.steps):
        solver.set_initial_guess(None)
        solver.set_initial_condition(h_u0)
        solver.solve()
        solver.solution(w["nt"] - 1, 1, out=h_out)
        hist = solver.residual_history()
    torch.cuda.synchronize(device)
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps
    e2e_ms = max_over_ranks(dist, e2e_ms, device)
    state_bytes = int(np.prod(shape)) * 8

    # rooflines of the event-timed level-0 propagator launch tables (every
    # state of one launch): the solver's level-0 sweeps (FP64, FP32) or, in
    # the refined modes, the FP64 residual pass and the FP32 inner cycles'
    # level-0 sweeps; `roofline` is the group with the larger share of the step
    refined = args.precision in ("fp32r", "fp32rf")
    fp64_rate = None
    if args.precision in ("fp64", "fp32r"):
        fp64_rate = atm.measure_fp64_rate(solver.stream)
    pk = peaks(fp64_rate)
    n_val = int(np.prod(shape))
    # states per profiled launch table: the level-0 relaxation launches cover
    # every interval; in the refined mode with full storage the FP64 pass
    # takes the residual of every time point
    jobs = {"allen_cahn_256": 256, "heat1d_127": 128, "allen_cahn_1024": 2048}[args.workload]
    if refined and args.storage == "full":
        jobs = w["nt"] - 1
    if args.algorithm == "seq":
        jobs = 1
    traffic_db = load_json(os.path.join(ROOT, "profiles", "traffic.json"), {}) or {}

    def stored_traffic(key, kind):
        tr = traffic_db.get(key)
        return tr["bytes_per_launch"] if tr and tr.get("source_hash") == kernel_source_hash(kind) else None

    def kernel_name(sc, what):
        k = sc["kernel"]
        if k in ("fused", "persistent"):
            kn = "fused_persist_kernel" if k == "persistent" else "fused_sweep_kernel"
            return (f"{kn} ({what}; cluster of {sc['ctas']} CTAs x {sc['threads']} threads, {sc['rows']}-row "
                    f"column segments" + (f", {sc['chunk']} resident clusters)" if k == "persistent" else ")"))
        if k == "float-float":
            return (f"df_sweep_kernel ({what}, float-float; cluster of {sc['ctas']} CTAs x {sc['threads']} "
                    f"threads, {sc['rows']}-row column segments)")
        if w["kind"] == "heat1d":
            return f"row_sweep_kernel ({what})"
        return f"row_sweep_kernel+col_sweep_kernel ({what}" + (
            f", {sc['chunk']} states per launch pair)" if sc.get("chunk") else ")")

    def roofline(which, sc, what, fp64_pipe, streams, desc, traffic_key, per_step_factor):
        tot = prof1[which][0] - prof0[which][0]
        cnt = prof1[which][1] - prof0[which][1]
        if cnt <= 0 or not tot > 0:
            return None
        avg = tot / cnt
        base = {"kernel": kernel_name(sc, what), "avg_launch_ms": avg, "launches_timed": cnt,
                "traffic": stored_traffic(traffic_key, sc["kernel"]),
                "share_of_step": tot / args.steps * per_step_factor / ms}
        if fp64_pipe:
            fpv = (FLOPS_PER_VALUE[("row", "heat1d")] if w["kind"] == "heat1d" else
                   FLOPS_PER_VALUE[("row", "pr_react")] + FLOPS_PER_VALUE[("col", "pr")])
            ach = fpv * n_val * jobs / (avg / 1e3) / 1e12
            return dict(base, bound="alu", achieved=ach, peak=pk["fp64_tflops"], unit="TFLOP/s",
                        frac=ach / pk["fp64_tflops"], peak_source=pk["fp64_src"],
                        frac_of_derived_peak=ach / FP64_DERIVED_TFLOPS,
                        algorithmic=f"{fpv} flop/value x {n_val} values x {jobs} states")
        nb = streams * n_val * jobs
        ach = nb / (avg / 1e3) / 1e9
        return dict(base, bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s", frac=ach / pk["hbm_gbs"],
                    peak_source=f"{pk['hbm_src']} STREAM copy (MEASURED_PEAKS.json)",
                    algorithmic=f"{desc} x {n_val} values x {jobs} states")

    if refined:
        sco = solver.sweep_config(-1)
        ff = args.precision == "fp32rf"
        r_outer = roofline(2, sco, "FP64 residual pass, level-0 propagator", not ff, 20,
                           "20 bytes per value (fp64 input, fp64 output, fp32 copy of the output)",
                           f"{args.workload}:{args.precision}:{args.storage}", 1.0)
        r_inner = roofline(3, solver.sweep_config(0), "FP32 inner cycles, level-0 propagator", False, 12,
                           "12 bytes per value (fp32 input, base of the increment, output)",
                           f"{args.workload}:fp32r_inner:{args.storage}",
                           float(args.inner_cycles or 5))
        cands = [r for r in (r_outer, r_inner) if r]
    else:
        fp64p = args.precision == "fp64"
        sb = 8 if args.precision in ("fp64", "fp64f") else 4
        cands = [r for r in [roofline(2, solver.sweep_config(0), "level-0 propagator", fp64p, 2 * sb,
                                      f"{2 * sb} bytes per value (input, output)",
                                      f"{args.workload}:{args.precision}:{args.storage}", 1.0)] if r]
    if not cands and w["kind"] == "heat1d" and args.sweep_kernel == "persistent":
        # the whole solve is one cooperative launch: its FP64 line-solve work
        # over the solve's time (propagator applications counted from the cycle)
        N0, m, k = w["nt"], w["m"][0], w["k"]
        NC = (N0 - 1) // m + 1
        nf = N0 - NC                                   # F-points
        coarse = NC - 1 if args.algorithm == "mgrit" else sum(min(p, k - 1) for p in range(NC))
        nu = w["nu"] if args.nu is None else args.nu
        it = int(np.median(iters))
        apps = nf + (NC - 1) + it * (nu * (NC - 1 + nf) + 2 * (NC - 1) + coarse + nf + (NC - 1))
        fpv = FLOPS_PER_VALUE[("row", "heat1d")]
        ach = fpv * n_val * apps / (ms / 1e3) / 1e12
        cands = [{"kernel": "persist1d_kernel (the whole solve, one cooperative launch)", "avg_launch_ms": ms,
                  "launches_timed": args.steps, "traffic": None, "share_of_step": 1.0, "bound": "alu",
                  "achieved": ach, "peak": pk["fp64_tflops"], "unit": "TFLOP/s", "frac": ach / pk["fp64_tflops"],
                  "peak_source": pk["fp64_src"],
                  "algorithmic": f"{fpv} flop/value x {n_val} values x {apps} propagator applications per solve"}]
    if not cands:
        raise RuntimeError("kernel profile recorded no launches")
    cands.sort(key=lambda r: -r["share_of_step"])
    roof = cands[0]
    roof_other = cands[1] if len(cands) > 1 else None
    if rank == 0:
        cpu, err = None, None
        if world == 1 and not args.no_cpu_baseline and args.workload != "allen_cahn_1024":
            cpu, cps = oracle_sequential_baseline(w, rank)
            err = error_vs_oracle(solver, w, cps)
            del cps
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "fp32r": "f32+f64", "fp64f": "f32x2",
                          "fp32rf": "f32+f32x2"}[args.precision],
                "data": "synthetic",
                "config": {"workload": args.workload,
                           **{k: (list(v) if isinstance(v, tuple) else v) for k, v in w.items()},
                           **({"nu": args.nu} if args.nu is not None else {}),
                           "algorithm": args.algorithm, "parallelism": f"{world} independent problems",
                           "sweep_kernel": args.sweep_kernel, "storage": args.storage, "nested": args.nested,
                           "cycle": "F" if args.fcycle else "V",
                           "inner_cycles": (args.inner_cycles or 5) if refined else None,
                           "inner_coarse_relax": args.inner_coarse_relax if refined else None,
                           "l2": "working set larger than L2 (workspace %.2f GB; one level-0 launch reads and "
                                 "writes %.0f MB)" % (atm.workspace_size(prob, desc) / 1e9,
                                                      2 * jobs * n_val * (4 if args.precision == "fp32" else 8) / 1e6)},
                "precision": args.precision,
                "iterations": int(np.median(iters)), "time_to_solution_ms": ms,
                "final_residual": float(res["final_residual"]),
                "residual_history": [float(v) for v in solver.residual_history()][:64],
                "e2e": {"value": world * (w["nt"] - 1) / (e2e_ms / 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes + 8 * len(hist)},
                "gpu_launches": int(launches),
                "coarse": args.coarse,
                "learned": None if learned_info is None else dict(
                    learned_info, fallback_in_timed_steps=sum(f for f, _, _ in fallbacks),
                    cycles_with_network_before_fallback=[i for _, i, _ in fallbacks],
                    residual_ending_the_network_attempt=[r for _, _, r in fallbacks]),
                "kernels_per_level": [solver.sweep_config(l) for l in range(len(w["m"]) + 1)]
                if args.algorithm != "seq" else [solver.sweep_config(0)],
                "roofline": roof, "roofline_other": roof_other, "cpu_baseline": cpu, "err_vs_oracle": err,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if args.tune_cache_out and rank == 0:
        with open(args.tune_cache_out, "w") as fh:
            fh.write(atm.tune_cache_export())
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
