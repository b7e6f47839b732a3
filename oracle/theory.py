"""Closed forms from the paper's two-level theory (Sec. 3) and the discrete
Fourier symbols of the propagators -- TEST INFRASTRUCTURE ONLY.

The symbols are the eigenvalues of the one-step operators on their Fourier
modes (the spatial matrices are normal, so Phi and Psi share eigenvectors and
Sec. 3.2's scalar analysis applies mode by mode).
"""
from __future__ import annotations

import numpy as np


def be_symbol_1d(j, D: float, dx: float):
    """Backward Euler on sin(j pi x) with Dirichlet second differences:
    1 / (1 + D (4/dx^2) sin^2(j pi dx / 2))."""
    j = np.asarray(j, dtype=np.float64)
    return 1.0 / (1.0 + D * (4.0 / dx ** 2) * np.sin(j * np.pi * dx / 2.0) ** 2)


def _sigma(q, n: int, h: float):
    """Eigenvalue magnitude of minus the periodic second difference on mode q."""
    q = np.asarray(q, dtype=np.float64)
    return (4.0 / h ** 2) * np.sin(np.pi * q / n) ** 2


def pr_symbol_2d(qx, qy, D: float, nx: int, ny: int, lx: float = 1.0, ly: float = 1.0):
    """Peaceman-Rachford ADI amplification: prod_d (1 - D/2 s_d) / (1 + D/2 s_d)."""
    sx, sy = _sigma(qx, nx, lx / nx), _sigma(qy, ny, ly / ny)
    return ((1 - 0.5 * D * sx) / (1 + 0.5 * D * sx)) * ((1 - 0.5 * D * sy) / (1 + 0.5 * D * sy))


def split_be_symbol_2d(qx, qy, D: float, nx: int, ny: int, lx: float = 1.0, ly: float = 1.0):
    """Split backward-Euler ADI amplification: 1 / ((1 + D s_x)(1 + D s_y))."""
    sx, sy = _sigma(qx, nx, lx / nx), _sigma(qy, ny, ly / ny)
    return 1.0 / ((1 + D * sx) * (1 + D * sy))


def ecc_matrix(lam: float, mu: float, m: int, k: int, npoints: int) -> np.ndarray:
    """Scalar C-to-C error propagator of two-level AT-MGRIT with F-relaxation
    (Sec. 3.2, the Toeplitz matrix for one eigenvalue pair): entry (p, q) is
    mu^x (lam^m - mu) on subdiagonal x + 1 for x = 0..k-2 and mu^(k-1) lam^m on
    subdiagonal k.  ``k >= npoints`` gives two-level MGRIT/Parareal."""
    E = np.zeros((npoints, npoints))
    lm = lam ** m
    for p in range(npoints):
        for q in range(p):
            d = p - q
            if d <= k - 1:
                E[p, q] = mu ** (d - 1) * (lm - mu)
            elif d == k:
                E[p, q] = mu ** (k - 1) * lm
    return E


def theorem1_bound(lam, mu, m: int, k: int):
    """Theorem 1: |lam^m - mu| (1 - |mu|^(k-1)) / (1 - |mu|) + |lam^m mu^(k-1)|."""
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    lm = lam ** m
    amu = np.abs(mu)
    geo = np.where(np.abs(1 - amu) > 1e-300, (1 - amu ** (k - 1)) / np.where(amu == 1, 1, 1 - amu), k - 1)
    return np.abs(lm - mu) * geo + np.abs(lm * mu ** (k - 1))


def dst_modes(nx: int) -> np.ndarray:
    """Orthonormal sine modes sin(j pi x_i) on the nx interior points
    (row j-1 holds mode j)."""
    x = np.arange(1, nx + 1) / (nx + 1)
    j = np.arange(1, nx + 1)[:, None]
    S = np.sin(np.pi * j * x[None, :])
    return S * np.sqrt(2.0 / (nx + 1))
