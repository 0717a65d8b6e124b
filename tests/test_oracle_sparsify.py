"""Pins of the oracle's sparsifying stencil and sparsified matrix C (Sec. 2), CPU only."""
import math

import numpy as np

from oracle import greens, sparsify
from paper_1602_07652_gb300 import inputs


def _setup(n=12, ppw=6.0):
    h = 1.0 / n
    w = inputs.omega_for_ppw(n, ppw)
    return n, h, w, sparsify.Stencils(n, h, w)


def test_C_equals_sparsified_product_A_H_brute_force():
    # Sec. 2: C is A H restricted to the 9-point pattern; dense A and H, n = 10.
    n, h, w, st = _setup(10)
    m = inputs.gaussian_disk_medium(n, amp=0.4, sigma=0.2, radius=0.45)
    A = sparsify.matrix_A(n, st).toarray()
    H = np.eye(n * n) + w * w * greens.dense_G(n, h, w) * m.ravel()[None, :]
    AH = A @ H
    C = sparsify.matrix_C(m, st, w).toarray()
    pattern = A != 0
    assert np.max(np.abs(np.where(pattern, AH, 0) - C)) < 1e-13 * np.max(np.abs(C))
    # off-pattern remainder: what sparsification drops; small next to the kept part
    off = np.linalg.norm(np.where(pattern, 0, AH)) / np.linalg.norm(AH)
    assert off < 0.2


def test_alpha_minimises_the_annihilation_problem():
    n, h, w, st = _setup(12)
    K = n
    W = greens.kernel_weights(K, h, w)
    rng = np.random.default_rng(0)
    for bx, bz in ((0, 0), (-1, 0), (0, 1), (1, -1)):
        slots = sparsify.stencil_slots(bx, bz)
        a = st.alpha[bz + 1, bx + 1]
        assert abs(np.linalg.norm(a) - 1) < 1e-13
        assert np.count_nonzero(a) == len(slots)
        c = a[sparsify.slot(0, 0)]
        assert abs(c.imag) < 1e-14 and c.real > 0
        # brute-force objective over the same window
        r = np.arange(-(n - 1), n)
        px = r if bx == 0 else (r[r >= 0] if bx == -1 else r[r <= 0])
        pz = r if bz == 0 else (r[r >= 0] if bz == -1 else r[r <= 0])
        PZ, PX = [x.ravel() for x in np.meshgrid(pz, px, indexing="ij")]
        inside = np.array([(abs(x) <= 1 and abs(z) <= 1 and sparsify.slot(x, z) in slots) for x, z in zip(PX, PZ)])
        PX, PZ = PX[~inside], PZ[~inside]

        def obj(v):
            s = 0
            for sl in slots:
                dx, dz = sparsify.OFFSETS[sl]
                s = s + v[sl] * W[dz - PZ + K, dx - PX + K]
            return np.linalg.norm(s)

        best = obj(a)
        for _ in range(50):
            v = np.zeros(9, complex)
            v[slots] = rng.standard_normal(len(slots)) + 1j * rng.standard_normal(len(slots))
            v /= np.linalg.norm(v)
            assert obj(v) >= best * (1 - 1e-12)
        # and small perturbations of alpha do not decrease it
        for _ in range(20):
            v = a.copy()
            v[slots] += 1e-4 * (rng.standard_normal(len(slots)) + 1j * rng.standard_normal(len(slots)))
            v /= np.linalg.norm(v)
            assert obj(v) >= best * (1 - 1e-12)


def test_stencils_respect_lattice_symmetry():
    # the square lattice is invariant under reflections and x <-> z; so are the minimisers
    n, h, w, st = _setup(12)
    A = st.alpha.reshape(3, 3, 3, 3)  # [bz, bx, dz, dx]
    tol = 1e-9
    assert np.max(np.abs(A[1, 1] - A[1, 1][::-1, :])) < tol          # interior: z-reflection
    assert np.max(np.abs(A[1, 1] - A[1, 1].T)) < tol                  # interior: x <-> z
    assert np.max(np.abs(A[0, 1] - A[2, 1][::-1, :])) < tol           # bottom edge = reflected top edge
    assert np.max(np.abs(A[1, 0] - A[0, 1].T)) < tol                  # left edge = transposed bottom edge
    assert np.max(np.abs(A[0, 0] - A[2, 2][::-1, ::-1])) < tol        # corners by reflection
    assert np.max(np.abs(A[0, 2] - A[0, 0][:, ::-1])) < tol
    tr = st.transposed()
    Ct = sparsify.matrix_C(np.zeros((n, n)), tr, w)
    C0 = sparsify.matrix_C(np.zeros((n, n)), st, w)
    # C of the transposed grid = P C P^T, P the x <-> z permutation
    perm = np.arange(n * n).reshape(n, n).T.ravel()
    assert abs(Ct - C0[perm][:, perm]).max() < tol


def test_zero_medium_C_is_A():
    n, h, w, st = _setup(8)
    C = sparsify.matrix_C(np.zeros((n, n)), st, w)
    A = sparsify.matrix_A(n, st)
    assert abs(C - A).max() == 0


def test_A_annihilates_G_away_from_the_stencil():
    # the point of A (Sec. 2): (A G)(k, p) is small for p outside mu(k)
    n, h, w, st = _setup(16, ppw=8.0)
    A = sparsify.matrix_A(n, st).toarray()
    G = greens.dense_G(n, h, w)
    AG = A @ G
    pattern = A != 0
    G_off = np.linalg.norm(np.where(pattern, 0, G))
    assert np.linalg.norm(np.where(pattern, 0, AG)) < 0.05 * G_off
