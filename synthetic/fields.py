"""Seeded synthetic magnetisation fields and surface charges.

Only random numbers and simple closed-form vector fields live here; nothing
in this module evaluates any part of the single layer potential.  The random
generator is numpy's PCG64 (``numpy.random.default_rng``), seeded per
workload so both the oracle and the CUDA path receive identical inputs.

Per-node fields are unit vectors at the mesh vertices (the P1 nodal values of
the paper's finite element magnetisation, Sec. 2.1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1305 * 100


def workload_seed(index: int) -> int:
    """Seed of workload ``index`` (cube 0, sphere 1, plate 2, batched 3, served 4)."""
    return SEED_BASE + int(index)


def _normalise(m):
    return m / np.linalg.norm(m, axis=1, keepdims=True)


def uniform(V, direction=(0.0, 0.0, 1.0)):
    """Uniform magnetisation (Sec. 4 sphere test uses m = e3)."""
    d = np.asarray(direction, dtype=np.float64)
    return np.tile(d / np.linalg.norm(d), (V.shape[0], 1))


def perturbed_uniform(V, seed, base=(1.0, 0.0, 0.0), amp=0.1):
    """base + U[-amp, amp]^3 per node, renormalised to |m| = 1 (cube workload)."""
    rng = np.random.default_rng(seed)
    m = np.asarray(base, dtype=np.float64)[None, :] + rng.uniform(-amp, amp, size=(V.shape[0], 3))
    return _normalise(m)


def vortex(V, seed, mz=0.3, noise=0.05):
    """(-y, x, mz)/norm plus N(0, noise^2) per component, renormalised (sphere workload)."""
    rng = np.random.default_rng(seed)
    m = np.stack([-V[:, 1], V[:, 0], np.full(V.shape[0], mz)], axis=1)
    m = _normalise(m)
    m = m + rng.normal(0.0, noise, size=m.shape)
    return _normalise(m)


def smooth_random(V, seed, n_modes=8, kmax=2):
    """Normalised sum of ``n_modes`` seeded low-frequency Fourier modes (plate workload).

    Each mode is a_j * cos(2 pi k_j . x_s + p_j) with k_j integer in
    [-kmax, kmax]^3 and x_s the node position scaled to the unit bounding box.
    """
    rng = np.random.default_rng(seed)
    lo = V.min(axis=0)
    ext = np.maximum(V.max(axis=0) - lo, 1e-30)
    xs = (V - lo) / ext
    m = np.zeros_like(V)
    for _ in range(n_modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        a = rng.normal(size=3)
        p = rng.uniform(0, 2 * np.pi)
        m += a[None, :] * np.cos(2 * np.pi * (xs @ k) + p)[:, None]
    m += 1e-3 * rng.normal(size=m.shape)  # keeps every node away from |m| = 0
    return _normalise(m)


def random_sigma(n_points, seed, lo=-1.0, hi=1.0):
    """Surface charge per quadrature point, uniform in [lo, hi] (Sec. 3.2 experiment)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n_points)


def random_mag(n_points, seed):
    """Random unit vectors per quadrature point."""
    rng = np.random.default_rng(seed)
    return _normalise(rng.normal(size=(n_points, 3)))
