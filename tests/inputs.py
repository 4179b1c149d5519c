"""Seeded synthetic inputs for the oracle pins and the CUDA-path parity tests.

This module holds none of the method's arithmetic: it only draws seeded random
numbers and builds hand-placed configurations (vortex lines, plane waves, gauge
functions).  Both sides of every parity test receive the arrays it returns.

Arrays have shape (10, N, N, N) in the plane order
  Re phi, Im phi, Re Pi, Im Pi, theta_x, theta_y, theta_z, E_x, E_y, E_z
indexed [plane, z, y, x] (x fastest), float64.
"""
from __future__ import annotations

import numpy as np


def perturbed_state(N: int, seed: int, sigma: float = 1.0, amp_phi: float = 0.3,
                    amp_pi: float = 0.3, amp_theta: float = 0.3, amp_e: float = 0.3) -> np.ndarray:
    """Random fields of moderate amplitude: phi = sigma (1 + a r) e^{i vartheta} with a
    uniformly random phase, Pi, theta, E uniform in [-amp, amp]."""
    rng = np.random.default_rng(seed)
    F = np.zeros((10, N, N, N))
    ph = rng.uniform(0.0, 2.0 * np.pi, (N, N, N))
    r = sigma * (1.0 + amp_phi * rng.uniform(-1.0, 1.0, (N, N, N)))
    F[0] = r * np.cos(ph)
    F[1] = r * np.sin(ph)
    F[2:4] = rng.uniform(-amp_pi, amp_pi, (2, N, N, N))
    F[4:7] = rng.uniform(-amp_theta, amp_theta, (3, N, N, N))
    F[7:10] = rng.uniform(-amp_e, amp_e, (3, N, N, N))
    return F


def smooth_state(N: int, seed: int, sigma: float = 1.0, amp: float = 0.05, kmax: int = 2) -> np.ndarray:
    """Vacuum plus a few long-wavelength random Fourier modes of small amplitude in
    every field (a configuration whose evolution stays smooth)."""
    rng = np.random.default_rng(seed)
    F = np.zeros((10, N, N, N))
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    F[0] = sigma
    for plane in range(10):
        for _ in range(3):
            k = rng.integers(-kmax, kmax + 1, 3)
            ph = rng.uniform(0, 2 * np.pi)
            F[plane] += amp * rng.uniform(0.5, 1.0) * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) / N + ph)
    return F


def gauge_function(N: int, seed: int) -> np.ndarray:
    """A random gauge function chi(x) uniform in [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, (N, N, N))


def vortex_pair_phase(N: int) -> np.ndarray:
    """Phase of a straight vortex (+1) / antivortex (-1) pair along z, cores at the
    plaquette centres (N/4 + 1/2, N/2 + 1/2) and (3N/4 + 1/2, N/2 + 1/2)."""
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    x1, y1 = N / 4 + 0.5, N / 2 + 0.5
    x2, y2 = 3 * N / 4 + 0.5, N / 2 + 0.5
    return np.arctan2(y - y1, x - x1) - np.arctan2(y - y2, x - x2)


def vortex_pair_cores(N: int):
    """Lower-left lattice corners (x, y) of the two plaquettes each z-layer's cores pierce."""
    return (N // 4, N // 2), (3 * N // 4, N // 2)


def square_loop_phase(N: int, R: int) -> np.ndarray:
    """Phase of a planar square string loop of side L = 2R in the plane z = N/2 + 1/2,
    edges on the dual lattice (half-integer x, y), centred at (N/2 + 1/2, N/2 + 1/2):
    vartheta = atan2(z - zc, r - R) with r the Chebyshev distance to the loop axis."""
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    c = N / 2 + 0.5
    r = np.maximum(np.abs(x - c), np.abs(y - c))
    return np.arctan2(z - c, r - R)


def branch_cut_phase(N: int, seed: int, eps: float = 2e-6) -> np.ndarray:
    """Phase pi (x + y) plus a uniform jitter in [-eps, eps] (N even): the phase
    difference across every x and y link lies within 2 eps of +-pi, the branch cut
    of arg, so the side each one lands on -- and with it most windings -- is decided
    at the cut."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return np.pi * (x + y) + rng.uniform(-eps, eps, (N, N, N))


def with_phase(theta: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """State with phi = sigma e^{i theta} and every other field zero."""
    N = theta.shape[0]
    F = np.zeros((10, N, N, N))
    F[0] = sigma * np.cos(theta)
    F[1] = sigma * np.sin(theta)
    return F


def plane_wave_coords(N: int):
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return x, y, z


def to_f32(F: np.ndarray) -> np.ndarray:
    """Round a float64 state to float32 (the engine's storage precision)."""
    return np.ascontiguousarray(F, dtype=np.float32)
