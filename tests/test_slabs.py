"""Time-slab decomposition (Sec. 4.1, Fig. 3) on the CPU: the plan of
paper_2107_09596_gb300.slabs, and a prototype of the distributed AT-MGRIT
cycle on 2 and 3 gloo ranks that follows it -- each rank holds its slab of
every level, the stages exchange exactly the plan's halo states (the last
point of the previous rank, the k - 1 coarse points before the rank's first
one) and the norm is one scalar all-reduce.  The prototype computes with the
oracle's propagators in the oracle's operation order, so its iterates must
equal the one-process oracle solve bit for bit (the norm's summation order
differs: residual histories to 1e-13)."""
import os
import socket

import numpy as np
import pytest

import atm_inputs as I
from paper_2107_09596_gb300.slabs import SlabPlan, level_points


def test_plan_covers_every_point_once_and_cuts_on_coarsest_points():
    for nt, m, world in ((130, (4, 2), 2), (130, (4, 2), 3), (4097, (16, 16), 8), (65, (4,), 5)):
        p = SlabPlan(nt, m, 3, world)
        for l in range(p.L):
            pts = [i for r in range(world) for i in p.owned(l, r)]
            assert pts == list(range(level_points(nt, m, l)))
        S = int(np.prod(m))
        for r in range(1, world):
            assert p.cuts[r] % S == 0
            for l in range(p.L - 1):
                # every rank starts with a C-point of every non-coarsest level
                assert p.lo[l][r] % m[l] == 0


def test_coarsest_halo_reaches_back_k_minus_1_points_over_several_ranks():
    p = SlabPlan(65, (4,), 6, 5)          # 17 coarse points over 5 ranks: 3 or 4 each
    l = p.L - 1
    for r in range(1, 5):
        got = [j for t in p.coarsest_halo() if t.dst == r for j in range(t.start, t.stop)]
        assert got == list(range(max(0, p.lo[l][r] - 5), p.lo[l][r]))
        for t in p.coarsest_halo():
            if t.dst == r:
                assert all(p.owner(l, j) == t.src for j in range(t.start, t.stop))
    # rank 4's window (5 points) spans ranks 2 and 3
    assert {t.src for t in p.coarsest_halo() if t.dst == 4} == {2, 3}
    assert p.bytes_per_cycle(8) > 0


def test_plan_rejects_more_ranks_than_coarsest_intervals():
    with pytest.raises(ValueError):
        SlabPlan(33, (4, 4), 2, 3)     # 2 coarsest intervals of 16 steps
    with pytest.raises(ValueError):
        SlabPlan(33, (4,), 0, 2)       # plain MGRIT has no slab plan


# ---------------------------------------------------------------------------
# the distributed cycle (test infrastructure: oracle propagators, numpy, gloo)
# ---------------------------------------------------------------------------
class SlabCycle:
    def __init__(self, dist, plan, c, u0):
        import oracle
        self.o, self.dist, self.p, self.c = oracle, dist, plan, c
        self.rank = dist.get_rank()
        shape = oracle.state_shape(c)
        self.L = plan.L
        self.u = [np.zeros((plan.N[l],) + shape) for l in range(self.L)]
        self.g = [None] + [np.zeros((plan.N[l],) + shape) for l in range(1, self.L)]
        self.v = [None] + [np.zeros((plan.N[l],) + shape) for l in range(1, self.L)]
        self.r = [None] + [np.zeros((plan.N[l],) + shape) for l in range(1, self.L)]
        self.g0 = u0.copy()
        self.u[0][0] = u0

    # exchange of states [start, stop) of an array, as the plan's transfers say
    def send_recv(self, transfers, arrays):
        import torch
        reqs, bufs = [], []
        for t in transfers:
            for a in arrays:
                if t.src == self.rank:
                    reqs.append(self.dist.isend(torch.from_numpy(np.ascontiguousarray(a[t.start:t.stop])), t.dst))
                elif t.dst == self.rank:
                    b = torch.empty(a[t.start:t.stop].shape, dtype=torch.float64)
                    reqs.append(self.dist.irecv(b, t.src))
                    bufs.append((a, t, b))
        for q in reqs:
            q.wait()
        for a, t, b in bufs:
            a[t.start:t.stop] = b.numpy()

    def phi(self, l, x):
        return self.o.apply_prop(self.c, l, x[None])[0]

    def rhs(self, l, j):
        if l > 0:
            return self.g[l][j]
        return self.g0 if j == 0 else None

    def step(self, l, j, src):
        t = self.phi(l, src)
        g = self.rhs(l, j)
        return t + g if g is not None else t

    def cpoints(self, l):
        m = self.c.m[l]
        return [i for i in range(0, self.p.N[l], m) if self.p.lo[l][self.rank] <= i < self.p.hi[l][self.rank]]

    def f_relax(self, l):
        m, N = self.c.m[l], self.p.N[l]
        for i0 in self.cpoints(l):
            for j in range(i0 + 1, min(i0 + m, N)):
                self.u[l][j] = self.step(l, j, self.u[l][j - 1])

    def c_relax(self, l):
        self.send_recv(self.p.neighbour_halo(l), [self.u[l]])
        for i0 in self.cpoints(l):
            if i0 == 0:
                self.u[l][0] = self.rhs(l, 0)
            else:
                self.u[l][i0] = self.step(l, i0, self.u[l][i0 - 1])

    def c_residual(self, l):
        """Residual at this rank's C-points of level l (coarse index -> state)."""
        self.send_recv(self.p.neighbour_halo(l), [self.u[l]])
        m, out = self.c.m[l], {}
        for i0 in self.cpoints(l):
            if i0 == 0:
                out[0] = self.rhs(l, 0) - self.u[l][0]
            else:
                out[i0 // m] = self.step(l, i0, self.u[l][i0 - 1]) - self.u[l][i0]
        return out

    def restrict(self, l):
        m, C = self.c.m[l], l + 1
        for i, ri in self.c_residual(l).items():
            self.r[C][i] = ri
            self.v[C][i] = self.u[l][i * m]
        self.send_recv(self.p.neighbour_halo(C), [self.v[C]])
        for i in self.p.owned(C, self.rank):
            if i == 0:
                self.g[C][0] = self.v[C][0] + self.r[C][0]
            else:
                t = self.phi(C, self.v[C][i - 1])
                self.g[C][i] = (self.v[C][i] - t) + self.r[C][i]
        own = self.p.owned(C, self.rank)
        self.u[C][own.start:own.stop] = self.v[C][own.start:own.stop]

    def coarsest(self):
        l, k = self.L - 1, self.c.k
        self.send_recv(self.p.coarsest_halo(), [self.v[l], self.r[l], self.g[l]])
        for p_ in self.p.owned(l, self.rank):
            j0 = max(0, p_ - k + 1)
            w = self.v[l][j0] + self.r[l][j0]
            for j in range(j0 + 1, p_ + 1):
                w = self.step(l, j, w)
            self.u[l][p_] = w

    def correct(self, l):
        m, C = self.c.m[l], l + 1
        for i in self.p.owned(C, self.rank):
            self.u[l][i * m] = self.u[l][i * m] + (self.u[C][i] - self.v[C][i])

    def cycle(self, l=0):
        if l == self.L - 1:
            self.coarsest()
            return
        self.f_relax(l)
        for _ in range(self.c.nu):
            self.c_relax(l)
            self.f_relax(l)
        self.restrict(l)
        self.cycle(l + 1)
        self.correct(l)
        self.f_relax(l)

    def norm(self):
        import torch
        s = sum(float(np.sum(r * r)) for r in self.c_residual(0).values())
        t = torch.tensor([s], dtype=torch.float64)
        self.dist.all_reduce(t)
        return float(np.sqrt(t.item()))


CASES = {
    "heat1d_2lvl": dict(kind="heat1d", nx=15, nt=130, m=(4,), k=5, nu=1),
    "ac_3lvl_fcf": dict(kind="ac", nx=16, ny=16, nt=130, m=(4, 2), k=3, nu=1),
    "ac_3lvl_f_k1": dict(kind="ac", nx=16, ny=16, nt=129, m=(2, 4), k=1, nu=0),
}


def _worker(rank, world, port, case, cycles, q):
    try:
        import torch.distributed as dist
        import oracle
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        kw = CASES[case]
        kind = {"heat1d": oracle.HEAT1D, "ac": oracle.ALLEN_CAHN}[kw["kind"]]
        c = oracle.make_cfg(kind, kw["nx"], kw.get("ny", 1), dt=1e-4 if kw["kind"] == "ac" else 1 / 256,
                            nt=kw["nt"], m=kw["m"], k=kw["k"], nu=kw["nu"],
                            react_exact=[l > 0 for l in range(len(kw["m"]) + 1)])
        shape = oracle.state_shape(c)
        u0 = I.uniform_field(shape, 41) if kw["kind"] == "ac" else I.heat1d_initial_condition(kw["nx"], 41)
        plan = SlabPlan(kw["nt"], kw["m"], kw["k"], world)
        sc = SlabCycle(dist, plan, c, u0)
        sc.f_relax(0)
        hist = [sc.norm()]
        for _ in range(cycles):
            sc.cycle()
            hist.append(sc.norm())
        # the one-process oracle solve of the same problem
        ref = np.zeros((kw["nt"],) + shape)
        ref[0] = u0
        _, rh = oracle.solve(c, ref, cycles, 0.0)
        own = plan.owned(0, rank)
        same = bool(np.array_equal(sc.u[0][own.start:own.stop], ref[own.start:own.stop]))
        hist_ok = bool(np.allclose(hist, rh, rtol=1e-13, atol=0))
        q.put((rank, same, hist_ok, hist, list(rh)))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, False, False, repr(e), None))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_distributed_cycle_equals_the_one_process_solve(case, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, 3, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for rank, same, hist_ok, hist, rh in res:
        assert same, (case, world, rank, hist)
        assert hist_ok, (case, world, rank, hist, rh)
