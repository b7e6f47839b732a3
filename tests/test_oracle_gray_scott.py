"""Pins of the oracle's Gray-Scott propagator (Sec. 5.1: backward Euler,
central differences, Newton's method per step) and of the space-time cycle on
that problem, against what the mathematics fixes independently of the
oracle's code: the reaction ODE of a spatially constant state (a separate
root finder), the Fourier symbols of the linearisation about the steady state
(u, v) = (1, 0), the backward Euler equation evaluated with an FFT Laplacian,
the sequential fixed point, exactness and the k >= N_T + 1 reduction.  CPU only."""
import numpy as np
import pytest
from scipy.optimize import fsolve

import atm_inputs as I

PAR = dict(du=8e-5, dv=4e-5, feed=0.024, kill=0.06)
DT = 256.0 / 16383.0          # 16384 points on [0, 256]


def gs_cfg(orc, nx=16, ny=16, lx=2.5, ly=2.5, dt=DT, nt=33, m=(4,), k=2, nu=0,
           tol=1e-12, fcycle=False):
    return orc.make_cfg(orc.GRAY_SCOTT, nx, ny, lx=lx, ly=ly, dt=dt, nt=nt, m=m, k=k, nu=nu,
                        fcycle=fcycle, gs=dict(PAR, tol=tol, max_iter=50))


def reaction(u, v, feed, kill):
    return -u * v * v + feed * (1 - u), u * v * v - (kill + feed) * v


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("D", [DT, 1.0, 16.0])
def test_constant_state_follows_the_reaction_ode(orc, D):
    # the Laplacian annihilates constants: Phi of a constant state is the
    # backward Euler step of the 2x2 reaction ODE, found here by fsolve
    c = gs_cfg(orc, nx=8, ny=8, dt=D, nt=3, m=(2,))
    states = []
    pairs = [(1.0, 0.0), (0.5, 0.25), (0.3, 0.4), (0.9, 0.05)]
    for u, v in pairs:
        s = np.empty((2, 8, 8))
        s[0], s[1] = u, v
        states.append(s)
    got = orc.apply_prop(c, 0, np.stack(states))
    for (u0, v0), g in zip(pairs, got):
        def eq(w):
            ru, rv = reaction(w[0], w[1], PAR["feed"], PAR["kill"])
            return [w[0] - u0 - D * ru, w[1] - v0 - D * rv]
        w = fsolve(eq, [u0, v0], xtol=1e-14)
        assert np.ptp(g[0]) < 1e-14 and np.ptp(g[1]) < 1e-14
        np.testing.assert_allclose([g[0, 0, 0], g[1, 0, 0]], w, rtol=0, atol=1e-12)


def test_linearisation_about_the_steady_state(orc):
    # (1, 0) is a steady state; the derivative of Phi there acts on each
    # Fourier mode of u by 1 / (1 + D (Du lam + F)) and of v by
    # 1 / (1 + D (Dv lam + K + F)), lam the symbol of -Lap.  nx != ny and
    # lx != ly so that a swapped axis fails; central difference in eps.
    nx, ny, lx, ly, D = 12, 8, 2.5, 1.7, 2.0
    c = gs_cfg(orc, nx=nx, ny=ny, lx=lx, ly=ly, dt=D, nt=3, m=(2,), tol=1e-14)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    modes = [(1, 2), (3, 1)]
    pu = np.cos(2 * np.pi * (modes[0][0] * x / nx + modes[0][1] * y / ny))
    pv = np.sin(2 * np.pi * (modes[1][0] * x / nx + modes[1][1] * y / ny))
    base = np.stack([np.ones((ny, nx)), np.zeros((ny, nx))])
    eps = 1e-4
    dirn = np.stack([pu, pv])
    out = orc.apply_prop(c, 0, np.stack([base + eps * dirn, base - eps * dirn]))
    deriv = (out[0] - out[1]) / (2 * eps)
    dx, dy = lx / nx, ly / ny

    def lam(kx, ky):
        return 4 / dx ** 2 * np.sin(np.pi * kx / nx) ** 2 + 4 / dy ** 2 * np.sin(np.pi * ky / ny) ** 2

    gu = 1 / (1 + D * (PAR["du"] * lam(*modes[0]) + PAR["feed"]))
    gv = 1 / (1 + D * (PAR["dv"] * lam(*modes[1]) + PAR["kill"] + PAR["feed"]))
    np.testing.assert_allclose(deriv[0], gu * pu, rtol=0, atol=1e-7)
    np.testing.assert_allclose(deriv[1], gv * pv, rtol=0, atol=1e-7)


@pytest.mark.parametrize("D", [DT, 1.0])
def test_step_solves_the_backward_euler_equation(orc, D):
    # residual of the step evaluated with the FFT symbol of the periodic
    # five-point Laplacian (a different route to the same operator)
    nx, ny, lx, ly = 16, 8, 2.5, 2.0
    c = gs_cfg(orc, nx=nx, ny=ny, lx=lx, ly=ly, dt=D, nt=3, m=(2,), tol=1e-12)
    w0 = I.gray_scott_random_state(nx, ny, seed=5)
    w = orc.apply_prop(c, 0, w0[None])[0]
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    sym = ((2 * np.cos(2 * np.pi * kx[None, :] / nx) - 2) / (lx / nx) ** 2
           + (2 * np.cos(2 * np.pi * ky[:, None] / ny) - 2) / (ly / ny) ** 2)

    def lap(f):
        return np.real(np.fft.ifft2(np.fft.fft2(f) * sym))

    ru, rv = reaction(w[0], w[1], PAR["feed"], PAR["kill"])
    Gu = w[0] - w0[0] - D * (PAR["du"] * lap(w[0]) + ru)
    Gv = w[1] - w0[1] - D * (PAR["dv"] * lap(w[1]) + rv)
    assert np.sqrt(np.sum(Gu ** 2) + np.sum(Gv ** 2)) < 1e-11
    assert np.abs(w - w0).max() > 1e-3          # the step did move the state


def test_newton_tolerance_is_met_and_counted(orc):
    c = gs_cfg(orc, nx=16, ny=16, dt=2.0, nt=3, m=(2,), tol=1e-10)
    gs = c.gray_scott
    n0, s0 = gs.newton_iterations, gs.steps
    x = np.stack([I.gray_scott_random_state(16, 16, seed=s) for s in range(3)])
    orc.apply_prop(c, 0, x)
    assert gs.steps - s0 == 3 and gs.failures == 0
    assert 3 <= gs.newton_iterations - n0 <= 3 * 12


def test_at_mgrit_converges_to_sequential(orc):
    c = gs_cfg(orc, nt=33, m=(4,), k=3, nu=1, tol=1e-13)
    u0 = I.gray_scott_initial_condition(16, 16)
    seq = orc.sequential(c, u0)
    u = np.zeros_like(seq)
    u[0] = u0
    it, hist = orc.solve(c, u, max_iter=20, tol=1e-11)
    assert hist[-1] <= 1e-11 and it < 20
    np.testing.assert_allclose(u, seq, rtol=0, atol=1e-11)


def test_exactness_after_j_iterations(orc):
    # two-level F-relaxation with a deliberately poor coarse grid (k = 1: no
    # coarse propagation at all): after j iterations the C-points 0..j equal
    # the sequential solution (the nonlinear solves' tolerance aside)
    c = gs_cfg(orc, nt=25, m=(4,), k=1, nu=0, tol=1e-13)
    u0 = I.gray_scott_initial_condition(16, 16)
    seq = orc.sequential(c, u0)
    for j in (1, 2, 3):
        u = np.zeros_like(seq)
        u[0] = u0
        orc.solve(c, u, max_iter=j)
        err = [np.abs(u[4 * i] - seq[4 * i]).max() for i in range(7)]
        assert max(err[: j + 1]) < 1e-12, (j, err)
        assert err[j + 1] > 1e-8, (j, err)


def test_large_k_is_mgrit(orc):
    nt, m = 33, 4
    nc = (nt - 1) // m + 1
    u0 = I.gray_scott_initial_condition(16, 16)
    res = []
    for k in (nc, 0):
        c = gs_cfg(orc, nt=nt, m=(m,), k=k, nu=1)
        u = np.zeros((nt, 2, 16, 16))
        u[0] = u0
        orc.solve(c, u, max_iter=2)
        res.append(u)
    assert np.array_equal(res[0], res[1])


def test_fcycle_with_two_levels_is_the_v_cycle(orc):
    # with two levels the coarse problem is solved directly (local grids), so
    # an F-cycle and a V-cycle are the same cycle, operation for operation
    u0 = I.gray_scott_initial_condition(16, 16)
    res = []
    for fc in (False, True):
        c = gs_cfg(orc, nt=33, m=(4,), k=3, nu=1, fcycle=fc)
        u = np.zeros((33, 2, 16, 16))
        u[0] = u0
        _, hist = orc.solve(c, u, max_iter=2)
        res.append((u, hist))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_nested_guess_two_levels_is_the_coarse_local_grid_solve(orc):
    # two levels: the nested start is the coarsest level solved by its local
    # grids from the guess (u0, 0, ..) (Sec. 2.2 nested iteration with the
    # local grids of Sec. 5.1).  The grid of point p starts at p - k + 1 from
    # v + r there; for p <= k that start is u0 or Psi(u0), so points 0..k are
    # the coarse sequential solution; later grids start from Psi(0), not from
    # the solution.
    nt, m, k = 33, 4, 3
    c = gs_cfg(orc, nt=nt, m=(m,), k=k, nu=1)
    u0 = I.gray_scott_initial_condition(16, 16)
    u = np.zeros((nt, 2, 16, 16))
    u[0] = u0
    orc.nested_guess(c, u)
    # the coarse sequential solution with step m dt
    cc = gs_cfg(orc, dt=m * DT, nt=(nt - 1) // m + 1, m=(2,), k=1)
    seq = orc.sequential(cc, u0)
    for p in range(k + 1):
        np.testing.assert_allclose(u[p * m], seq[p], rtol=0, atol=1e-11)
    assert np.abs(u[(k + 1) * m] - seq[k + 1]).max() > 1e-6


def test_line_search_carries_newton_through_a_hard_step(orc):
    # a large step from an unstructured state: full Newton steps overshoot by
    # orders of magnitude (first trial ~1e6 against ||G|| ~ 3); the halving
    # line search keeps every accepted residual below the previous one until
    # the quadratic phase, and the step meets the tolerance
    from oracle.gray_scott import GrayScott
    gs = GrayScott(16, 16, 2.5, 2.5, tol=1e-12, max_iter=60, **PAR)
    w0 = I.gray_scott_random_state(16, 16, seed=9).ravel()
    D = 3.0
    trials = []
    orig = gs.be_residual

    def record(w, w_prev, DD):
        G = orig(w, w_prev, DD)
        trials.append(np.linalg.norm(G))
        return G

    gs.be_residual = record
    w = gs.step(w0, D)
    assert gs.failures == 0 and np.linalg.norm(orig(w, w0, D)) <= 1e-12
    assert max(trials) > 1e5 * trials[0]            # full steps do overshoot
    assert gs.newton_iterations > 5                  # and the search is what carries it
