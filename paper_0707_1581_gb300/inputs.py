"""Seeded synthetic inputs shared by the tests and the benchmark.

Only random or analytic fields live here -- no lattice weights, no
equilibrium, nothing of the method's arithmetic -- so the CUDA path and the
FP64 oracle can be fed the same inputs without sharing code.  Every generator
is a pure function of its arguments (numpy PCG64 with the given seed).
"""
from __future__ import annotations

import numpy as np


def relative_perturbation(shape, seed: int, amp: float, ncomp: int = 19) -> np.ndarray:
    """Factors 1 + amp * N(0, 1) of shape [ncomp, *shape]; multiplied by the
    populations of a rest state they give a state with small random density,
    momentum, stress and kinetic content."""
    rng = np.random.default_rng(seed)
    return 1.0 + amp * rng.standard_normal((ncomp,) + tuple(shape))


def smooth_velocity(shape, seed: int, amp: float, nmodes: int = 4) -> np.ndarray:
    """u[3, nz, ny, nx]: a sum of `nmodes` Fourier modes with small integer wave
    numbers and random phases per component, scaled to max |u_alpha| ~ amp."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3,) + tuple(shape))
    for a in range(3):
        for _ in range(nmodes):
            k = rng.integers(-2, 3, 3)
            ph = rng.uniform(0, 2 * np.pi)
            u[a] += np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + ph)
    return amp * u / nmodes


def shear_wave(shape, u0: float) -> np.ndarray:
    """u = (u0 sin(2 pi z / nz), 0, 0): the transverse wave whose decay gives
    the shear viscosity."""
    nz, ny, nx = shape
    u = np.zeros((3,) + tuple(shape))
    u[0] = u0 * np.sin(2 * np.pi * np.arange(nz) / nz)[:, None, None]
    return u


def sample_sites(nsites_total: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct site indices in [0, nsites_total), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nsites_total, size=min(count, nsites_total), replace=False)).astype(np.int64)


def mixed_edges(n: int = 16, lo: int = 32, hi: int = 128, step: int = 8) -> list[int]:
    """Edges of `n` cubic boxes spread evenly from lo to hi in multiples of step."""
    return [lo + step * int(round((hi - lo) / step * j / (n - 1))) for j in range(n)]


def uniform_draws(n: int, seed: int, lo: float, hi: float) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, n)
