"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module draws media, incident angles and random fields only. It holds none
of the method's arithmetic (no kernel, quadrature, stencil or solver), so both
sides can take their inputs from it without sharing any computation.

Grid convention (Sec. 2 of the paper): nodes x_{i,j} = (h i, h j) with
1 <= i <= n_x, 1 <= j <= n_z and h = 1/n.  Arrays are indexed [j-1, i-1]
(z slow, x fast), i.e. row-major with x contiguous, matching the ordering
v = (v_1, ..., v_{n_z}), v_j = (v_{1,j}, ..., v_{n_x,j}) of Sec. 3.2.
"""
from __future__ import annotations

import numpy as np


def node_coords(n: int):
    """Return (X, Z) arrays of shape (n, n) with X[j, i] = (i+1)/n, Z[j, i] = (j+1)/n."""
    h = 1.0 / n
    c = h * np.arange(1, n + 1, dtype=np.float64)
    Z, X = np.meshgrid(c, c, indexing="ij")
    return X, Z


def gaussian_disk_medium(n: int, amp: float = -0.2, sigma: float = 0.1,
                         radius: float = 0.3, center=(0.5, 0.5)) -> np.ndarray:
    """m = amp * exp(-|x-c|^2 / (2 sigma^2)) on the disk |x-c| <= radius, else 0."""
    X, Z = node_coords(n)
    r2 = (X - center[0]) ** 2 + (Z - center[1]) ** 2
    m = amp * np.exp(-r2 / (2.0 * sigma * sigma))
    m[r2 > radius * radius] = 0.0
    return m


def bump_medium(n: int, nbumps: int = 20, seed: int = 0, support: float = 0.4,
                sigma_range=(0.02, 0.08), amp_range=(-0.3, 0.3),
                center=(0.5, 0.5)) -> np.ndarray:
    """Sum of seeded Gaussian bumps supported in the disk |x-c| <= support.

    sigma_b ~ U[sigma_range], a_b ~ U[amp_range], bump centres uniform in the
    disk of radius support - 2 sigma_b; the sum is cut to the disk.
    """
    rng = np.random.default_rng(seed)
    X, Z = node_coords(n)
    m = np.zeros((n, n), dtype=np.float64)
    for _ in range(nbumps):
        s = rng.uniform(*sigma_range)
        a = rng.uniform(*amp_range)
        rmax = max(support - 2.0 * s, 0.0)
        rr = rmax * np.sqrt(rng.uniform())
        ph = rng.uniform(0.0, 2.0 * np.pi)
        cx = center[0] + rr * np.cos(ph)
        cz = center[1] + rr * np.sin(ph)
        m += a * np.exp(-((X - cx) ** 2 + (Z - cz) ** 2) / (2.0 * s * s))
    r2 = (X - center[0]) ** 2 + (Z - center[1]) ** 2
    m[r2 > support * support] = 0.0
    return m


def constant_disk_medium(n: int, m0: float, radius: float,
                         center=(0.5, 0.5)) -> np.ndarray:
    """Piecewise-constant contrast m0 on the closed disk |x-c| <= radius."""
    X, Z = node_coords(n)
    r2 = (X - center[0]) ** 2 + (Z - center[1]) ** 2
    return np.where(r2 <= radius * radius, m0, 0.0).astype(np.float64)


def smooth_medium(n: int, amp: float = 0.2, width: float = 0.12,
                  center=(0.5, 0.5)) -> np.ndarray:
    """A C-infinity compactly supported bump: amp*exp(1 - 1/(1-(r/w)^2)) for r < w."""
    X, Z = node_coords(n)
    r2 = ((X - center[0]) ** 2 + (Z - center[1]) ** 2) / (width * width)
    m = np.zeros((n, n), dtype=np.float64)
    inside = r2 < 1.0
    m[inside] = amp * np.exp(1.0 - 1.0 / (1.0 - r2[inside]))
    return m


def seeded_angle(seed: int = 0) -> float:
    """One incident direction theta ~ U[0, 2 pi) from the given seed."""
    return float(np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi))


def random_field(n: int, seed: int, nz: int | None = None) -> np.ndarray:
    """Seeded complex field (nz x n) with i.i.d. standard normal real/imag parts."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nz, n)) + 1j * rng.standard_normal((nz, n))


def omega_for_ppw(n: int, ppw: float) -> float:
    """Frequency giving `ppw` points per wavelength on the unit square, h = 1/n."""
    return 2.0 * np.pi * n / ppw
