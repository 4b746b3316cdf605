"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module draws random numbers only; it holds none of the method's
arithmetic.  The draws follow one counter-based generator, SplitMix64
(S. Vigna's published finaliser with the golden-ratio increment), keyed by
(seed, field id, site index):

    x = seed XOR (field << 40) XOR (y * nx + x_site)
    z = x + 0x9E3779B97F4A7C15   (mod 2^64)
    z = (z XOR (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z XOR (z >> 27)) * 0x94D049BB133111EB
    z =  z XOR (z >> 31)
    U = (z >> 11) * 2^-53            in [0, 1)

The CUDA library implements the same definition independently for its
on-device initialiser, so both sides draw identical numbers.

Field ids: 0 = concentration perturbation, 1 = director angle.
"""
from __future__ import annotations

import numpy as np

FIELD_PHI = 0
FIELD_THETA = 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counter values x (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, field: int, nx: int, ny: int) -> np.ndarray:
    """U[0, 1) draws of shape (ny, nx) for one (seed, field) stream."""
    idx = np.arange(nx * ny, dtype=np.uint64)
    key = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(field) << np.uint64(40)) ^ idx
    z = splitmix64(key)
    return ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53).reshape(ny, nx)


def initial_draws(seed: int, nx: int, ny: int):
    """The two draws of the initial condition: (U_phi, U_theta), each (ny, nx).

    The initial condition takes phi = phi0 + dphi (2 U_phi - 1) and a director
    angle theta = pi U_theta; converting them to Q is each side's own work.
    """
    return uniform01(seed, FIELD_PHI, nx, ny), uniform01(seed, FIELD_THETA, nx, ny)


def random_field(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Generic seeded normal field for tests (numpy PCG64 stream)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
