"""Pins of the oracle's one-step propagators against independent definitions:
dense linear algebra, Fourier symbols and the reaction ODE.  CPU only."""
import math

import numpy as np
import pytest

import atm_inputs as I
from oracle import theory as T


def lap1d_dirichlet(n, h):
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = -2.0
        if i > 0:
            L[i, i - 1] = 1.0
        if i < n - 1:
            L[i, i + 1] = 1.0
    return L / h ** 2


def lap1d_periodic(n, h):
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = -2.0
        L[i, (i - 1) % n] += 1.0
        L[i, (i + 1) % n] += 1.0
    return L / h ** 2


def test_heat1d_be_matches_dense_solve(orc):
    n, lx, D = 13, 1.7, 0.003
    c = orc.make_cfg(orc.HEAT1D, n, lx=lx, dt=D, nt=5, m=(2,))
    h = lx / (n + 1)
    A = np.eye(n) - D * lap1d_dirichlet(n, h)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, n))
    got = orc.apply_prop(c, 0, x)
    want = np.linalg.solve(A, x.T).T
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("pr", [True, False])
def test_adi2d_matches_dense_kronecker(orc, pr):
    # nx != ny and lx != ly so that a swapped axis or a transposed operand fails
    nx, ny, lx, ly, D = 7, 5, 1.0, 1.3, 0.002
    prop = orc.PROP_PR if pr else orc.PROP_SPLIT
    c = orc.make_cfg(orc.HEAT2D, nx, ny, lx=lx, ly=ly, dt=D, nt=5, m=(2,), prop=[prop, prop])
    Lx = lap1d_periodic(nx, lx / nx)
    Ly = lap1d_periodic(ny, ly / ny)
    Ix, Iy = np.eye(nx), np.eye(ny)
    # state u[y][x] flattened with x fastest: operator along x is kron(Iy, Lx)
    KX, KY = np.kron(Iy, Lx), np.kron(Ly, Ix)
    I2 = np.eye(nx * ny)
    if pr:
        M = np.linalg.solve(I2 - 0.5 * D * KY, I2 + 0.5 * D * KX) @ \
            np.linalg.solve(I2 - 0.5 * D * KX, I2 + 0.5 * D * KY)
    else:
        M = np.linalg.inv(I2 - D * KY) @ np.linalg.inv(I2 - D * KX)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, ny, nx))
    got = orc.apply_prop(c, 0, x).reshape(3, -1)
    want = (M @ x.reshape(3, -1).T).T
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_heat1d_fourier_symbol(orc):
    n, D = 31, 1.0 / 64
    c = orc.make_cfg(orc.HEAT1D, n, dt=D, nt=5, m=(4,))
    S = T.dst_modes(n)
    lam = T.be_symbol_1d(np.arange(1, n + 1), D, 1.0 / (n + 1))
    out = orc.apply_prop(c, 0, S)
    np.testing.assert_allclose(out, lam[:, None] * S, rtol=1e-12, atol=1e-13)
    # coarse level: step m*D
    out1 = orc.apply_prop(c, 1, S)
    mu = T.be_symbol_1d(np.arange(1, n + 1), 4 * D, 1.0 / (n + 1))
    np.testing.assert_allclose(out1, mu[:, None] * S, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("pr", [True, False])
def test_adi2d_fourier_symbol(orc, pr):
    nx, ny, D = 16, 12, 2e-3
    prop = orc.PROP_PR if pr else orc.PROP_SPLIT
    c = orc.make_cfg(orc.HEAT2D, nx, ny, dt=D, nt=5, m=(2,), prop=[prop, prop])
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for qx, qy in [(0, 0), (1, 0), (0, 1), (3, 5), (8, 6), (7, 2)]:
        mode = np.cos(2 * math.pi * (qx * xx / nx + qy * yy / ny))
        out = orc.apply_prop(c, 0, mode[None])[0]
        sym = (T.pr_symbol_2d if pr else T.split_be_symbol_2d)(qx, qy, D, nx, ny)
        np.testing.assert_allclose(out, sym * mode, rtol=1e-12, atol=1e-13)


def test_allen_cahn_constant_field_follows_reaction(orc):
    # the periodic Laplacian annihilates constants: Phi(c) is the reaction alone
    n, D, eps = 8, 1e-4, 0.02
    c = orc.make_cfg(orc.ALLEN_CAHN, n, n, dt=D, nt=33, eps=eps, m=(4, 2))
    for val in (-0.7, 0.0, 0.3, 1.0):
        u = np.full((1, n, n), val)
        out = orc.apply_prop(c, 0, u)
        want = val + D * (val - val ** 3) / eps ** 2
        np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-15)
        # level 1 (split-BE, 4 substeps of the fine step) and level 2 (8 substeps)
        for lev, s in ((1, 4), (2, 8)):
            w = val
            for _ in range(s):
                w = w + D * (w - w ** 3) / eps ** 2
            out = orc.apply_prop(c, lev, u)
            np.testing.assert_allclose(out, w, rtol=1e-12, atol=1e-15)


def test_allen_cahn_odd_symmetry(orc):
    n = 12
    c = orc.make_cfg(orc.ALLEN_CAHN, n, n, dt=1e-4, nt=33, eps=0.02, m=(4, 2))
    u = I.uniform_field((2, n, n), 7, -0.9, 0.9)
    for lev in (0, 1, 2):
        a = orc.apply_prop(c, lev, u)
        b = orc.apply_prop(c, lev, -u)
        np.testing.assert_array_equal(a, -b)


def test_allen_cahn_reaction_then_adi(orc):
    # Lie splitting: Phi = ADI(reaction(u)); check against the heat2d ADI applied
    # to an explicitly reacted field
    n, D, eps = 10, 1e-4, 0.05
    ca = orc.make_cfg(orc.ALLEN_CAHN, n, n, dt=D, nt=5, eps=eps, m=(2,))
    ch = orc.make_cfg(orc.HEAT2D, n, n, dt=D, nt=5, eps=eps, m=(2,))
    u = I.uniform_field((1, n, n), 11, -1, 1)
    w = u + D * (u - u ** 3) / eps ** 2
    np.testing.assert_allclose(orc.apply_prop(ca, 0, u), orc.apply_prop(ch, 0, w),
                               rtol=1e-14, atol=1e-15)


def test_exact_reaction_flow_against_fine_euler(orc):
    """The exact flow of u' = (u - u^3)/eps^2 used on coarse levels agrees with
    a very fine explicit Euler integration of the same ODE (first order in the
    substep), on constant fields where the diffusion acts as the identity."""
    n, D, eps = 8, 1e-4, 0.02
    c_exact = orc.make_cfg(orc.ALLEN_CAHN, n, n, dt=D, nt=33, eps=eps, m=(4, 2),
                           react_exact=[0, 1, 1])
    for val in (-0.9, -0.05, 0.0, 0.01, 0.5, 1.0):
        u = np.full((1, n, n), val)
        for lev, steps in ((1, 4), (2, 8)):
            out = orc.apply_prop(c_exact, lev, u)[0, 0, 0]
            Dl = steps * D
            errs = []
            for s in (20000, 40000):
                w = val
                for _ in range(s):
                    w = w + (Dl / s) * (w - w ** 3) / eps ** 2
                errs.append(abs(w - out))
            assert errs[1] <= 5e-5 * max(1.0, abs(out))
            if errs[0] > 1e-12:
                assert 1.6 < errs[0] / errs[1] < 2.4     # first-order convergence to the flow
