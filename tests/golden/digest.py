"""Compact digest of a large field, for comparing a GPU field with a stored oracle field.

A 2048 x 2048 complex field is 64 MB; what is stored instead (by make_oracle_digests.py,
which runs only the oracle) is
  * a seeded subsampled randomized Fourier sketch  s(u) = sqrt(N/k) (F (d * u))[I]:
    d random signs, F the unitary 2-D DFT, I k random frequencies.  E ||s(e)||^2 = ||e||^2
    for any e, and the random signs spread every e over all frequencies, so
    ||s(u) - s(u*)|| / ||u*|| estimates the relative L2 error of u to about 1/sqrt(2k)
    of itself (k = 2048: about 2 %);
  * the field's values at seeded random grid points (compared one by one);
  * ||u*||_2 and max |u*|.
No method arithmetic lives here: the sketch is a measurement, applied identically to the
oracle's field and to the field under test.
"""
from __future__ import annotations

import numpy as np

SKETCH_K = 2048
SKETCH_SEED = 20160225
POINT_SEED = 777
POINT_COUNT = 1024


def _signs_and_freqs(n: int, seed: int, k: int):
    rng = np.random.default_rng(seed)
    d = rng.choice(np.array([-1.0, 1.0]), size=(n, n))
    idx = rng.choice(n * n, size=k, replace=False)
    return d, idx


def sketch(u: np.ndarray, seed: int = SKETCH_SEED, k: int = SKETCH_K) -> np.ndarray:
    """s(u) = sqrt(N/k) (F (d * u))[I], F the unitary 2-D DFT (k complex numbers)."""
    n = u.shape[0]
    d, idx = _signs_and_freqs(n, seed, k)
    Fu = np.fft.fft2(d * u, norm="ortho").ravel()
    return np.sqrt(n * n / k) * Fu[idx]


def points(n: int, seed: int = POINT_SEED, count: int = POINT_COUNT):
    """Seeded grid points (j, i) (row j = z index, column i = x index)."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(n * n, size=count, replace=False)
    return np.stack([flat // n, flat % n], axis=1)


def make(u: np.ndarray) -> dict:
    n = u.shape[0]
    s = sketch(u)
    pts = points(n)
    vals = u[pts[:, 0], pts[:, 1]]
    return {"n": n, "norm": float(np.linalg.norm(u)), "max_abs": float(np.abs(u).max()),
            "sketch_k": SKETCH_K, "sketch_seed": SKETCH_SEED, "sketch": [[float(z.real), float(z.imag)] for z in s],
            "point_seed": POINT_SEED, "points": pts.tolist(),
            "values": [[float(z.real), float(z.imag)] for z in vals]}


def compare(u: np.ndarray, dg: dict) -> dict:
    """Estimated relative L2 error of u against the digested field, and the largest
    pointwise error at the stored points relative to max |u*|."""
    ref_s = np.array([complex(a, b) for a, b in dg["sketch"]])
    s = sketch(u, dg["sketch_seed"], dg["sketch_k"])
    pts = np.array(dg["points"])
    ref_v = np.array([complex(a, b) for a, b in dg["values"]])
    v = u[pts[:, 0], pts[:, 1]]
    return {"rel_l2_est": float(np.linalg.norm(s - ref_s) / dg["norm"]),
            "max_rel_points": float(np.abs(v - ref_v).max() / dg["max_abs"]),
            "norm_ratio": float(np.linalg.norm(u) / dg["norm"])}
