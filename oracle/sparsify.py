"""Oracle: sparsifying preconditioner A and the sparsified matrix C (Sec. 2).

Test infrastructure only (see oracle/__init__.py).  FP64 throughout.

Paper passages followed (Sec. 2, "sparsifying preconditioner")
  * mu(k) = {p : ||k - p||_inf <= 1, x_p in Omega}: the 3 x 3 stencil, clipped
    at the boundary of Omega.
  * A(k, mu(k)) nonzero only; A(k, :) G(:, mu(k)^c) ~ 0, A translation invariant;
    alpha minimises ||alpha G(mu(0), mu(0)^c)|| over ||alpha|| = 1, by SVD.
  * C = A H thresholded to the pattern of A; the inner system is C u = A f
    (eq. preconditioner; eq. global_sparse_system).

Readings
  * The printed formula for alpha is garbled.  alpha is the conjugate of the left
    singular vector of G(mu(0), mu(0)^c) for its smallest singular value: with
    M = U S V^*, ||alpha M|| = ||S U^T alpha^T|| is minimised by alpha = conj(U[:, -1]).
    Its phase is free; we make the centre coefficient real and positive (C and
    g = A f scale together, so C^{-1} A f does not depend on it).
  * mu(0)^c is taken over all offsets p of the grid relative to the centre:
    the window [-(n-1), n-1]^2 minus the stencil.
  * Boundary points (the paper defers them to Ying's Sec. 4): a point on an edge
    of Omega has the 6-point stencil mu(k) (offsets leaving Omega dropped) and a
    corner the 4-point one; each of the 9 types (bx, bz) in {-1, 0, 1}^2 solves
    its own SVD problem over the window clipped to the half-plane / quadrant
    that stays inside Omega.
  * Sparsification: (A H)(k, k+d) for d in mu(k) is
        alpha_d + w^2 beta_d m_{k+d},  beta_d = sum_{e in mu(k)} alpha_e G_w(e - d),
    which is what C keeps (entries of A H off the pattern are dropped).
Stencil slot s = (dz + 1) * 3 + (dx + 1) for offset d = (dx, dz).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps

from . import greens

OFFSETS = [(dx, dz) for dz in (-1, 0, 1) for dx in (-1, 0, 1)]


def slot(dx: int, dz: int) -> int:
    return (dz + 1) * 3 + (dx + 1)


def stencil_slots(bx: int, bz: int):
    """Slots of mu(k) for a point of type (bx, bz): offsets that stay inside Omega."""
    out = []
    for s, (dx, dz) in enumerate(OFFSETS):
        if (bx == -1 and dx == -1) or (bx == 1 and dx == 1):
            continue
        if (bz == -1 and dz == -1) or (bz == 1 and dz == 1):
            continue
        out.append(s)
    return out


def point_type(i: int, n: int) -> int:
    """-1 on the first grid line, +1 on the last one, 0 inside."""
    return -1 if i == 0 else (1 if i == n - 1 else 0)


def sparsifying_stencil(n: int, h: float, omega: float, bx: int = 0, bz: int = 0,
                        W: np.ndarray | None = None) -> np.ndarray:
    """alpha for stencil type (bx, bz): a length-9 vector (zeros off mu) (Sec. 2, SVD problem).

    W, if given, is greens.kernel_weights(n, h, omega) (the same table for every type).
    """
    slots = stencil_slots(bx, bz)
    K = n  # offsets d - p reach |.| <= n
    if W is None:
        W = greens.kernel_weights(K, h, omega)
    rng = np.arange(-(n - 1), n)
    px = rng if bx == 0 else (rng[rng >= 0] if bx == -1 else rng[rng <= 0])
    pz = rng if bz == 0 else (rng[rng >= 0] if bz == -1 else rng[rng <= 0])
    PZ, PX = np.meshgrid(pz, px, indexing="ij")
    PX = PX.ravel()
    PZ = PZ.ravel()
    keep = ~((np.abs(PX) <= 1) & (np.abs(PZ) <= 1)
             & np.isin(slot_vec(PX, PZ), slots))
    PX = PX[keep]
    PZ = PZ[keep]
    M = np.empty((len(slots), PX.size), dtype=np.complex128)
    for a, s in enumerate(slots):
        dx, dz = OFFSETS[s]
        M[a] = W[dz - PZ + K, dx - PX + K]
    U, S, Vh = np.linalg.svd(M, full_matrices=False)
    a = np.conj(U[:, -1])
    c = a[slots.index(slot(0, 0))]
    a = a * (np.conj(c) / abs(c))
    alpha = np.zeros(9, dtype=np.complex128)
    alpha[slots] = a
    return alpha


def slot_vec(dx, dz):
    return (np.asarray(dz) + 1) * 3 + (np.asarray(dx) + 1)


def beta_table(alpha: np.ndarray, bx: int, bz: int, h: float, omega: float) -> np.ndarray:
    """beta_d = sum_{e in mu} alpha_e G_w(e - d) for d in mu (Sec. 2: (A G)(k, k+d))."""
    slots = stencil_slots(bx, bz)
    W = greens.kernel_weights(2, h, omega)
    beta = np.zeros(9, dtype=np.complex128)
    for sd in slots:
        dx, dz = OFFSETS[sd]
        acc = 0j
        for se in slots:
            ex, ez = OFFSETS[se]
            acc += alpha[se] * W[ez - dz + 2, ex - dx + 2]
        beta[sd] = acc
    return beta


class Stencils:
    """alpha and beta tables for the 9 point types, indexed [bz + 1][bx + 1]."""

    def __init__(self, n: int, h: float, omega: float):
        self.n, self.h, self.omega = n, h, omega
        self.alpha = np.zeros((3, 3, 9), dtype=np.complex128)
        self.beta = np.zeros((3, 3, 9), dtype=np.complex128)
        W = greens.kernel_weights(n, h, omega)  # one table of G_w serves the 9 SVD problems
        for bz in (-1, 0, 1):
            for bx in (-1, 0, 1):
                a = sparsifying_stencil(n, h, omega, bx, bz, W)
                self.alpha[bz + 1, bx + 1] = a
                self.beta[bz + 1, bx + 1] = beta_table(a, bx, bz, h, omega)

    def transposed(self) -> "Stencils":
        """Tables for the transposed grid (x <-> z): type and offset swap roles."""
        t = object.__new__(Stencils)
        t.n, t.h, t.omega = self.n, self.h, self.omega
        t.alpha = np.zeros_like(self.alpha)
        t.beta = np.zeros_like(self.beta)
        for bz in range(3):
            for bx in range(3):
                for s, (dx, dz) in enumerate(OFFSETS):
                    st = slot(dz, dx)
                    t.alpha[bx, bz, st] = self.alpha[bz, bx, s]
                    t.beta[bx, bz, st] = self.beta[bz, bx, s]
        return t


def assemble(m_coef: np.ndarray, st: Stencils, omega: float, types_z=None, types_x=None,
             with_m: bool = True) -> sps.csr_matrix:
    """Sparse matrix with entries alpha_d + w^2 beta_d m_{k+d} on mu(k) (Sec. 2: C; A if with_m=False).

    m_coef: (nz, nx) coefficient field; types_z / types_x: the type of each row /
    column line (default: the boundary of the array is the boundary of Omega).
    """
    nz, nx = m_coef.shape
    tz = np.array([point_type(j, nz) for j in range(nz)] if types_z is None else types_z)
    tx = np.array([point_type(i, nx) for i in range(nx)] if types_x is None else types_x)
    JJ, II = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    BZ = tz[JJ]
    BX = tx[II]
    rows, cols, vals = [], [], []
    for s, (dx, dz) in enumerate(OFFSETS):
        ok = ~(((BX == -1) & (dx == -1)) | ((BX == 1) & (dx == 1))
               | ((BZ == -1) & (dz == -1)) | ((BZ == 1) & (dz == 1)))
        j = JJ[ok]
        i = II[ok]
        v = st.alpha[BZ[ok] + 1, BX[ok] + 1, s]
        if with_m:
            v = v + omega * omega * st.beta[BZ[ok] + 1, BX[ok] + 1, s] * m_coef[j + dz, i + dx]
        rows.append(j * nx + i)
        cols.append((j + dz) * nx + (i + dx))
        vals.append(v)
    N = nz * nx
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))


def matrix_C(m: np.ndarray, st: Stencils, omega: float) -> sps.csr_matrix:
    """Sparsified matrix C (Sec. 2)."""
    return assemble(m, st, omega, with_m=True)


def matrix_A(n: int, st: Stencils) -> sps.csr_matrix:
    """Sparsifying matrix A: A(k, k+d) = alpha_d on mu(k) (Sec. 2)."""
    return assemble(np.zeros((n, n)), st, 0.0, with_m=False)


def apply_A(r: np.ndarray, st: Stencils) -> np.ndarray:
    n = r.shape[0]
    return (matrix_A(n, st) @ r.ravel()).reshape(r.shape)


def apply_C(v: np.ndarray, m: np.ndarray, st: Stencils, omega: float) -> np.ndarray:
    return (matrix_C(m, st, omega) @ v.ravel()).reshape(v.shape)
