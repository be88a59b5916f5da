"""Seeded synthetic initial fields for the benchmark problems of arXiv:1803.11345.

This module holds input generation only — none of the scheme's arithmetic — so that the
CUDA path and the CPU oracle can be fed the very same arrays.  Every generator returns
row-major (ny, nx) float64 arrays (index y * nx + x).

Random draws use the counter-based SplitMix64 generator (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): value k of stream ``seed`` is the
finaliser applied to seed + (k + 1) * 0x9E3779B97F4A7C15, so any element can be regenerated
independently of the others.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output number ``index`` (0-based) of the stream started at ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (index.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) with 53 random bits each."""
    z = splitmix64(seed, np.arange(count, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def interface_width(gamma: float, a: float) -> float:
    """sqrt(2) xi with xi = sqrt(gamma / a): the tanh length of a flat interface."""
    return math.sqrt(2.0 * gamma / a)


def droplet(nx: int, ny: int, R: float, gamma: float, a: float, cx: float | None = None,
            cy: float | None = None) -> np.ndarray:
    """Circular droplet of radius R (phi = +1 inside, -1 outside) with the tanh profile."""
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(x - cx, y - cy)
    return np.tanh((R - r) / interface_width(gamma, a))


def spinodal(nx: int, ny: int, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """phi i.i.d. uniform in [-amplitude, amplitude], element k = y * nx + x of the stream."""
    return (amplitude * (2.0 * uniform01(seed, nx * ny) - 1.0)).reshape(ny, nx)


def layers(nx: int, ny: int, y_lo: float, y_hi: float, gamma: float, a: float) -> np.ndarray:
    """A band phi = +1 for y_lo < y < y_hi (cell centres at y + 1/2), -1 outside, with tanh
    edges: two flat interfaces parallel to the x axis."""
    w = interface_width(gamma, a)
    y = np.arange(ny, dtype=np.float64) + 0.5
    prof = np.tanh((y - y_lo) / w) - np.tanh((y - y_hi) / w) - 1.0
    return np.repeat(prof[:, None], nx, axis=1)


def batch_members(count: int, seed: int):
    """Sizes, kinds and parameters of a batched sweep of independent lattices:
    nx in {64,128,256,512}, ny = nx or nx/2, half droplets and half spinodal, viscosity ratio
    log-uniform in [1, 1000], capillary number log-uniform in [0.01, 0.5]."""
    u = uniform01(seed, 6 * count).reshape(count, 6)
    sizes = np.array([64, 128, 256, 512])
    out = []
    for k in range(count):
        nx = int(sizes[min(3, int(u[k, 0] * 4))])
        ny = nx if u[k, 1] < 0.5 else nx // 2
        out.append(dict(nx=nx, ny=ny, kind="droplet" if u[k, 2] < 0.5 else "spinodal",
                        zeta=float(10.0 ** (3.0 * u[k, 3])),
                        Ca=float(10.0 ** (math.log10(0.01) + (math.log10(0.5) - math.log10(0.01)) * u[k, 4])),
                        seed=int(seed * 1000003 + k)))
    return out
