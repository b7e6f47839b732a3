"""Gray-Scott propagator of the oracle -- TEST INFRASTRUCTURE ONLY.

Sec. 5.1 of arXiv 2107.09596: two species on a periodic square,
    u_t = Du Lap u - u v^2 + F (1 - u),
    v_t = Dv Lap v + u v^2 - (K + F) v,
central differences in space (five-point Laplacian), backward Euler in time,
each step's nonlinear system solved by Newton's method with relative and
absolute tolerance `tol`.  The printed v equation has -(K+F)u; the decay
term of the model the paper cites removes v, and that reading is taken here.

One backward Euler step with step D maps w_prev to the root w of
    G(w) = w - w_prev - D (Lap_D w + R(w)),
found from w = w_prev by Newton iterations w <- w - lam * J(w)^-1 G(w) with
J(w) = I - D (Lap_D + dR/dw) solved exactly (sparse LU, a library
primitive), a halving line search on ||G||_2 (lam = 1, 1/2, ..., 1/1024;
the first lam with ||G(w - lam d)|| <= (1 - 1e-4 lam) ||G(w)||, else the
last one), stopped when ||G(w)||_2 <= max(tol, tol * ||G(w_prev)||_2) or
after `max_iter` iterations.

State layout: the u field (ny rows of nx values, x fastest), then the v
field, 2 nx ny values.
"""
from __future__ import annotations

import ctypes

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def periodic_second_difference(n: int, h: float):
    """(f_{i-1} - 2 f_i + f_{i+1}) / h^2 with indices modulo n."""
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    M = sp.diags([off, main, off], [-1, 0, 1], format="lil")
    M[0, n - 1] += 1.0
    M[n - 1, 0] += 1.0
    return M.tocsr() / (h * h)


class GrayScott:
    def __init__(self, nx, ny, lx, ly, du, dv, feed, kill, tol=1e-10, max_iter=50):
        self.nx, self.ny = nx, ny
        self.du, self.dv, self.feed, self.kill = du, dv, feed, kill
        self.tol, self.max_iter = tol, max_iter
        n = nx * ny
        self.n = n
        lap = (sp.kron(sp.identity(ny), periodic_second_difference(nx, lx / nx))
               + sp.kron(periodic_second_difference(ny, ly / ny), sp.identity(nx)))
        self.lap = lap.tocsr()
        # diffusion of the stacked state (u, v)
        self.diff = sp.block_diag([du * self.lap, dv * self.lap], format="csr")
        self.newton_iterations = 0
        self.steps = 0
        self.failures = 0

    def reaction(self, w):
        u, v = w[: self.n], w[self.n:]
        uvv = u * v * v
        return np.concatenate([-uvv + self.feed * (1.0 - u), uvv - (self.kill + self.feed) * v])

    def reaction_jacobian(self, w):
        u, v = w[: self.n], w[self.n:]
        return sp.bmat([[sp.diags(-v * v - self.feed), sp.diags(-2.0 * u * v)],
                        [sp.diags(v * v), sp.diags(2.0 * u * v - (self.kill + self.feed))]])

    def be_residual(self, w, w_prev, D):
        """G(w) = w - w_prev - D (Lap_D w + R(w))."""
        return w - w_prev - D * (self.diff @ w + self.reaction(w))

    def step(self, w_prev, D):
        """One backward Euler step by Newton's method (see the module text)."""
        w = np.array(w_prev, dtype=np.float64, copy=True)
        G = self.be_residual(w, w_prev, D)
        f = np.linalg.norm(G)
        stop = max(self.tol, self.tol * f)
        it = 0
        while f > stop and it < self.max_iter:
            J = (sp.identity(2 * self.n) - D * (self.diff + self.reaction_jacobian(w))).tocsc()
            d = sla.spsolve(J, G)
            lam = 1.0
            for h in range(11):
                wt = w - lam * d
                Gt = self.be_residual(wt, w_prev, D)
                ft = np.linalg.norm(Gt)
                if ft <= (1.0 - 1e-4 * lam) * f or h == 10:
                    break
                lam *= 0.5
            w, G, f = wt, Gt, ft
            it += 1
        self.newton_iterations += it
        self.steps += 1
        if f > stop:
            self.failures += 1
        return w


EXT_PROP = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_double,
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def make_callback(gs: GrayScott):
    """C callback out = Phi(in) for the oracle library (state of 2 nx ny values)."""
    size = 2 * gs.n

    def prop(level, D, pin, pout):
        out = np.ctypeslib.as_array(pout, shape=(size,))
        try:
            w_prev = np.ctypeslib.as_array(pin, shape=(size,)).copy()
            out[:] = gs.step(w_prev, D)
        except Exception:      # the C side cannot see a Python error: poison the result
            out[:] = np.nan

    return EXT_PROP(prop)
