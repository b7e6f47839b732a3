"""Time-slab decomposition of AT-MGRIT over several GPUs (Sec. 4.1, Fig. 3).

Host-side plan only: which time points each rank owns on every level of the
hierarchy and which states it must receive from other ranks before each stage
of a V-cycle (Algorithm 2).  The time axis is cut at multiples of the coarsest
spacing S = m_0 m_1 ... m_{L-2}, so that on every level a rank owns whole
intervals (a C-point and the F-points that follow it) and the ragged end of
the time grid belongs to the last rank.  With that cut the stages need:

  * F-relaxation: nothing (every interval is owned by one rank);
  * C-relaxation and the C-point residual of level l: the last point of the
    previous rank on level l (one state, neighbour send);
  * FAS right-hand side of level l + 1: the last injected point v of the
    previous rank on level l + 1 (one state, neighbour send);
  * local coarse grids of the coarsest level (the AT step): the k - 1 coarse
    points before the rank's first one (v, r and g of each), which is the
    paper's grouped exchange of the k - 1 preceding coarse residuals; when a
    rank owns fewer than k - 1 coarsest points the window reaches back over
    several ranks;
  * correction: nothing;
  * the residual norm: one scalar all-reduce (sum of squares).

Plain MGRIT's sequential coarsest solve has no such decomposition (it is a
chain through all ranks); the plan covers AT-MGRIT (k >= 1).
"""
from __future__ import annotations

from dataclasses import dataclass


def level_points(nt: int, m, level: int) -> int:
    """Points of level `level`: N_0 = nt, N_{l+1} = (N_l - 1) / m_l + 1."""
    n = nt
    for j in range(level):
        n = (n - 1) // m[j] + 1
    return n


def spacing(m, level: int) -> int:
    """Fine points per level-`level` step: m_0 ... m_{level-1}."""
    s = 1
    for j in range(level):
        s *= m[j]
    return s


@dataclass(frozen=True)
class Transfer:
    """States [start, stop) of a level that rank `src` sends to rank `dst`."""
    src: int
    dst: int
    level: int
    start: int
    stop: int


class SlabPlan:
    """Contiguous time slabs of `world` ranks for nt points, coarsening
    factors m (levels = len(m) + 1) and local grids of k points."""

    def __init__(self, nt: int, m, k: int, world: int):
        m = tuple(int(x) for x in m)
        if nt < 2 or not m or any(x < 2 for x in m):
            raise ValueError("need nt >= 2 and coarsening factors >= 2")
        if k < 1:
            raise ValueError("the slab plan covers AT-MGRIT (k >= 1)")
        self.nt, self.m, self.k, self.world = nt, m, k, world
        self.L = len(m) + 1
        S = spacing(m, self.L - 1)
        full = (nt - 1) // S        # coarsest intervals of S fine steps
        if world < 1 or world > full:
            raise ValueError(f"{world} ranks for {full} coarsest intervals")
        base, extra = divmod(full, world)
        cuts = [S * (r * base + min(r, extra)) for r in range(world)] + [nt]
        self.cuts = cuts            # rank r owns fine points [cuts[r], cuts[r + 1])
        self.N = [level_points(nt, m, l) for l in range(self.L)]
        # owned points per level: [lo, hi)
        self.lo = [[cuts[r] // spacing(m, l) for r in range(world)] for l in range(self.L)]
        self.hi = [[(cuts[r + 1] // spacing(m, l) if r + 1 < world else self.N[l]) for r in range(world)]
                   for l in range(self.L)]

    def owned(self, level: int, rank: int) -> range:
        return range(self.lo[level][rank], self.hi[level][rank])

    def owner(self, level: int, index: int) -> int:
        for r in range(self.world):
            if self.lo[level][r] <= index < self.hi[level][r]:
                return r
        raise IndexError(index)

    def neighbour_halo(self, level: int) -> list:
        """The last point of every rank on `level`, sent to the next rank (the
        C-relaxation, the C-point residual on `level`; for level >= 1 also the
        FAS right-hand side, which applies Psi to the previous injected point)."""
        return [Transfer(r - 1, r, level, self.lo[level][r] - 1, self.lo[level][r]) for r in range(1, self.world)]

    def coarsest_halo(self) -> list:
        """The k - 1 coarsest points before each rank's first one, split by
        owner (v, r and g of those points are sent)."""
        l = self.L - 1
        out = []
        for r in range(1, self.world):
            start = max(0, self.lo[l][r] - (self.k - 1))
            j = start
            while j < self.lo[l][r]:
                src = self.owner(l, j)
                stop = min(self.hi[l][src], self.lo[l][r])
                out.append(Transfer(src, r, l, j, stop))
                j = stop
        return out

    def bytes_per_cycle(self, state_bytes: int, nu: int = 1) -> int:
        """Bytes sent between ranks in one V-cycle (F(CF)^nu relaxation):
        per non-coarsest level (1 + nu) neighbour sends of a state (the
        C-relaxations and the residual) plus one for the FAS right-hand side of
        the next level, one more on level 0 for the residual of the stopping
        test; three states per coarsest-halo point; the norm's scalar
        all-reduce is not counted."""
        sends = len(self.neighbour_halo(0))
        for l in range(self.L - 1):
            sends += (1 + nu) * len(self.neighbour_halo(l)) + len(self.neighbour_halo(l + 1))
        halo = sum(t.stop - t.start for t in self.coarsest_halo())
        return state_bytes * (sends + 3 * halo)
