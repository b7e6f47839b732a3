"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path.

This module only draws numbers: it holds none of the method's arithmetic
(no propagator, no residual, no multigrid step).  Both sides receive the
arrays it returns as plain inputs.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to [0, 1) by taking the
top 53 bits.  The generator is written out here so that every machine draws
the same numbers for the same seed.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Return ``count`` successive splitmix64 outputs (uint64) for ``seed``."""
    out = np.empty(count, dtype=np.uint64)
    state = seed & _MASK
    for i in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1): top 53 bits of splitmix64 times 2**-53."""
    if count <= 4096:
        bits = splitmix64(seed, count)
    else:
        bits = _splitmix64_vec(seed, count)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _splitmix64_vec(seed: int, count: int) -> np.ndarray:
    """Vectorised splitmix64: the i-th output uses state seed + (i+1)*gamma."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def heat1d_initial_condition(nx: int, seed: int = 0, modes: int = 8,
                             amplitude: float = 0.1) -> np.ndarray:
    """u0(x) = sin(pi x) + amplitude * sum_j a_j sin(q_j pi x) on the nx interior
    points x_i = (i+1)/(nx+1) of [0, 1]; q_j uniform in {1..nx}, a_j uniform(-1, 1)."""
    r = uniform01(seed, 2 * modes)
    x = np.arange(1, nx + 1, dtype=np.float64) / (nx + 1)
    u = np.sin(math.pi * x)
    for j in range(modes):
        q = 1 + int(r[2 * j] * nx)
        a = 2.0 * r[2 * j + 1] - 1.0
        u = u + amplitude * a * np.sin(q * math.pi * x)
    return u


def uniform_field(shape, seed: int = 0, low: float = -0.05,
                  high: float = 0.05) -> np.ndarray:
    """A field of independent uniform(low, high) values (Allen-Cahn initial data)."""
    n = int(np.prod(shape))
    return (low + (high - low) * uniform01(seed, n)).reshape(shape)


def random_guess(nt: int, shape, seed: int = 1, low: float = -1.0,
                 high: float = 1.0) -> np.ndarray:
    """Space-time initial guess: uniform(low, high) at every time point (the
    caller keeps its own initial condition at t0)."""
    n = int(np.prod(shape))
    return (low + (high - low) * uniform01(seed, nt * n)).reshape((nt,) + tuple(shape))


def batch_problem_draws(count: int, seed: int = 0):
    """Draw the parameters of ``count`` independent problems for a batched run:
    kind in {heat2d, allen_cahn}, n in {64,128,256,512}, nt in {1025,4097,16385},
    m in {8,16}.  Returns a list of dicts of plain ints/strings."""
    r = uniform01(seed, 4 * count)
    kinds = ("heat2d", "allen_cahn")
    ns = (64, 128, 256, 512)
    nts = (1025, 4097, 16385)
    ms = (8, 16)
    out = []
    for i in range(count):
        out.append({
            "kind": kinds[int(r[4 * i] * 2)],
            "n": ns[int(r[4 * i + 1] * 4)],
            "nt": nts[int(r[4 * i + 2] * 3)],
            "m": ms[int(r[4 * i + 3] * 2)],
            "seed": i,
        })
    return out


def conv_net_init(seed: int = 0, channels=(1, 32, 32, 32, 32, 1)):
    """Seeded initial weights of a stack of 3x3 convolutions: layer l draws
    uniform(-b, b) with b = sqrt(6 / (9 c_in)) (He-style), the last layer scaled
    by 0.1 so that u + N(u) starts near the identity; biases zero.  Returns a
    list of (w [c_out][c_in][3][3], b [c_out]) float64 arrays."""
    params = []
    for li in range(len(channels) - 1):
        ci, co = channels[li], channels[li + 1]
        bound = np.sqrt(6.0 / (9 * ci))
        if li == len(channels) - 2:
            bound *= 0.1
        w = (2 * uniform01(seed + li, co * ci * 9) - 1).reshape(co, ci, 3, 3) * bound
        params.append((w, np.zeros(co)))
    return params


def gray_scott_initial_condition(nx: int, ny: int, lx: float = 2.5, ly: float = 2.5) -> np.ndarray:
    """The Gray-Scott initial state of Sec. 5.1 on the periodic grid
    x_i = i lx / nx, y_j = j ly / ny: inside the square [1, 1.5]^2,
    s = 0.25 sin^2(4 pi x) sin^2(4 pi y), u = 1 - 2 s, v = s; outside, u = 1,
    v = 0.  Shape (2, ny, nx): the u field, then the v field."""
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny)
    Y, X = np.meshgrid(y, x, indexing="ij")
    inside = (X >= 1.0) & (X <= 1.5) & (Y >= 1.0) & (Y <= 1.5)
    s = np.where(inside, 0.25 * np.sin(4 * np.pi * X) ** 2 * np.sin(4 * np.pi * Y) ** 2, 0.0)
    return np.ascontiguousarray(np.stack([1.0 - 2.0 * s, s]))


def gray_scott_random_state(nx: int, ny: int, seed: int = 0) -> np.ndarray:
    """A seeded state of the Gray-Scott ranges: u uniform in [0.2, 1], v
    uniform in [0, 0.45] (the ranges a run from the Sec. 5.1 initial state
    visits).  Shape (2, ny, nx)."""
    r = uniform01(seed, 2 * nx * ny).reshape(2, ny, nx)
    return np.ascontiguousarray(np.stack([0.2 + 0.8 * r[0], 0.45 * r[1]]))
