"""Training data for the learned coarse propagator from the method itself.

The coarse propagator Psi approximates m fine steps (Sec. 2.1, last
paragraph).  The states it meets in a solve are the C-point values of the
iterates of the first cycles, not only points of converged trajectories, so
the pairs here are the ones the method's own F-relaxation produces: after c
V-cycles from the zero guess, the level-0 C-points u_{(i-1)m} of the iterate,
and the values that an F-relaxation followed by a C-relaxation leaves at the
next C-points, u_{im} = Phi^m(u_{(i-1)m}) (level 0 has no right-hand side
after t_0).  Every step runs in the library (atm_solve, atm_run_stage,
atm_level_read); this module only sequences the calls and collects the
states.
"""
from __future__ import annotations

from . import ARRAY_U, STAGE_C_RELAX, STAGE_F_RELAX, Solver


def method_pairs(problem, make_desc, initial_conditions, cycles, device="cuda:0"):
    """Pairs (u_C, Phi^m u_C) from the F-relaxations of the first cycles.

    problem: the level-0 problem (atm_problem); make_desc(c): a solver
    description (MGRIT or AT-MGRIT, full level-0 storage, tol 0) that runs
    exactly c >= 1 cycles; initial_conditions: FP64 states (torch tensors on
    `device`); cycles: the cycle counts whose iterates give pairs.  Returns
    (inputs, targets): FP32 device tensors of shape (pairs, ny, nx), ordered
    by cycle count, initial condition and interval."""
    import torch
    ins, outs = [], []
    for c in cycles:
        if c < 1:
            raise ValueError("cycle counts start at 1")
        s = Solver(problem, make_desc(c), device=device)
        n, m = s.level_points(0), s.desc.m[0]
        cps = range(0, n, m)
        for u0 in initial_conditions:
            s.set_initial_guess(None)
            s.set_initial_condition(u0)
            s.solve()
            before = torch.cat([s.level_read(0, ARRAY_U, t, 1) for t in cps])
            s.run_stage(STAGE_F_RELAX, 0)
            s.run_stage(STAGE_C_RELAX, 0)
            after = torch.cat([s.level_read(0, ARRAY_U, t, 1) for t in cps])
            ins.append(before[:-1].to(torch.float32))
            outs.append(after[1:].to(torch.float32))
            del before, after
        s.close()
    return torch.cat(ins).contiguous(), torch.cat(outs).contiguous()
