"""Oracle: layered domain decomposition and the polarized-traces preconditioners.

Test infrastructure only (see oracle/__init__.py).  FP64 throughout.

Paper passages followed
  * Sec. 3.1: L horizontal layers Omega^l, each extended (Omega^l_ext); local
    problems C^l w^l = g^l = chi_{Omega^l} g (eq. local_discrete_sparse_pde);
    C^l equals C inside Omega^l (compatibility condition).
  * Sec. 3.2: ordering of unknowns (eq. global_ordering, eq. trace_ordering),
    traces v^l_0, v^l_1, v^l_n, v^l_{n+1}, discrete measure delta_k, and the
    discrete Green's representation formula (eq. pde_GRF_real).
  * Sec. 3.3: C^l built from D^l = diag(xi^l m) with a cut-off xi^l constant in x
    and a cubic spline in z, the stencil of the boundary of Omega on the outer
    rows of Omega^l_ext, and an O(w) complex shift in the cut-off region.
  * Sec. 3.4, eq. pde_GRF_down and Algorithm 1 (Gauss-Seidel preconditioner).
  * Sec. 3.5, Algorithm 2 (bi-directional preconditioner).
  * Sec. 4.1, local factorisations: the paper calls them "circulant"; read as
    banded (C^l is block tridiagonal in x-slow order), factored by a partial-
    pivoted sparse LU in that order (no fill-reducing column permutation).

Readings (the paper's displays for xi^l, delta_k and eq. local_discrete_sparse_pde
are empty in the available text, and Algorithm 1's layer indices are garbled)
  * Layers l = 0..L-1 from the bottom (small z) up; layer l owns global rows
    [l t, (l+1) t), t = n / L.  The extended strip has q = t + 2E rows, local row
    r <-> global row l t - E + r.  Local row "1" of the paper is r = E, row "0"
    is r = E-1, row "n^l" is r = E+t-1, row "n^l+1" is r = E+t.
  * A strip never extends past Omega: rows outside Omega are decoupled
    identity rows (so q stays uniform); the first and last rows inside Omega of
    every strip use the boundary stencil types (bz = -1 / +1).
  * xi^l = 1 on Omega^l and on the two halo rows 0 and n^l+1 (needed for the
    compatibility condition); over the remaining E-1 rows on each side it is
    the cubic S(tau) = 1 - 3 tau^2 + 2 tau^3, tau = (dist-1)/(E-1), reaching 0 on
    the outermost row (dist = number of rows beyond the layer).
  * Complex shift: C^l uses m^l = xi^l m + i (c / w) (1 - xi^l), i.e. an added
    i c w in the w^2-weighted coefficient where the cut-off is below one.
  * (delta_k p)_{i,j} = p_i on local row k, 0 elsewhere.
  * Algorithm 1, downward sweep l = L-1..0: layer l receives from layer l+1
    (eq. pde_GRF_down): g^l += -delta_{n} C^l_{n,n+1} w^{l+1}_1
    + delta_{n+1} C^l_{n+1,n} w^{l+1}_0.  Upward sweep l = 0..L-1 keeps that g^l
    and receives from layer l-1 through the same formula at its bottom rows,
    g^l += -delta_1 C^l_{1,0} p_0 + delta_0 C^l_{0,1} p_1, with the up-going
    traces p_0 = v^{l-1}_n - w^l_0 and p_1 = v^{l-1}_{n+1}.  The pair injected must
    be the traces of one wave field: the top injection of layer l-1 reproduces
    the down-going wave in its row n but cancels it in its extension row n+1, so
    the literal pair (v^{l-1}_n, v^{l-1}_{n+1}) carries the down-going wave in one
    row only and acts as a spurious source (a point source in the top layer is
    then reproduced with O(1) error).  Removing that wave from row n -- it is
    w^l_0, the continuation of layer l's own down-sweep solution below it --
    leaves the up-going field, which is what the upward sweep transmits (Sec. 3.4:
    polarized traces).  Output: interior rows of v^l.
  * "Preconditioner^T" in Algorithm 2 is Algorithm 1 on vertical layers, i.e. on
    the grid with x and z exchanged (the left-right pass of Sec. 3.5).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import sparsify


def cutoff(dist: int, E: int) -> float:
    """xi as a function of the number of rows beyond the layer (reading above)."""
    if dist <= 1:
        return 1.0
    tau = (dist - 1) / (E - 1)
    return 1.0 - 3.0 * tau * tau + 2.0 * tau ** 3


class Layering:
    """Horizontal layered decomposition of an (n_z, n_x) grid (Sec. 3.1)."""

    def __init__(self, m: np.ndarray, st: sparsify.Stencils, omega: float, L: int,
                 E: int = 10, shift: float = 10.0):
        nz, nx = m.shape
        if nz % L:
            raise ValueError("L must divide n_z")
        self.m, self.st, self.omega, self.L, self.E, self.shift = m, st, omega, L, E, shift
        self.nz, self.nx = nz, nx
        self.t = nz // L
        self.q = self.t + 2 * E
        self.layers = [self._build(l) for l in range(L)]

    def row_global(self, l: int, r: int) -> int:
        return l * self.t - self.E + r

    def _build(self, l: int):
        t, q, E, nx, nz = self.t, self.q, self.E, self.nx, self.nz
        zs = [self.row_global(l, r) for r in range(q)]
        real = [0 <= z < nz for z in zs]
        r_lo = real.index(True)
        r_hi = q - 1 - real[::-1].index(True)
        mcoef = np.zeros((q, nx), dtype=np.complex128)
        types_z = []
        for r, z in enumerate(zs):
            if not real[r]:
                types_z.append(0)
                continue
            if z < l * t:
                dist = l * t - z
            elif z >= (l + 1) * t:
                dist = z - (l + 1) * t + 1
            else:
                dist = 0
            xi = cutoff(dist, E)
            mcoef[r] = xi * self.m[z] + 1j * (self.shift / self.omega) * (1.0 - xi)
            types_z.append(-1 if r == r_lo else (1 if r == r_hi else 0))
        # assemble on the real rows, identity on the padding rows
        Creal = sparsify.assemble(mcoef[r_lo:r_hi + 1], self.st, self.omega, types_z=types_z[r_lo:r_hi + 1])
        blocks = []
        if r_lo > 0:
            blocks.append(sps.identity(r_lo * nx, dtype=np.complex128))
        blocks.append(Creal)
        if r_hi < q - 1:
            blocks.append(sps.identity((q - 1 - r_hi) * nx, dtype=np.complex128))
        Cl = sps.block_diag(blocks, format="csc")
        # Banded LU (Sec. 4.1 "local factorisation"): unknowns reordered x-slow, so C^l is
        # block tridiagonal with q x q blocks (band q + 1 each side); partial-pivoted LU in
        # that natural order keeps the fill inside the band.
        perm = np.arange(q * nx).reshape(q, nx).T.ravel()   # x-slow index (i, r) -> r nx + i
        lu = spla.splu(Cl[perm][:, perm].tocsc(), permc_spec="NATURAL")
        return dict(C=Cl, lu=lu, perm=perm, mcoef=mcoef, types_z=types_z, real=real)

    # -- blocks of C^l between two local rows, applied to a trace (Sec. 3.2) --
    def coupling(self, l: int, r_from: int, r_to: int, p: np.ndarray) -> np.ndarray:
        """(C^l_{r_from, r_to} p)_i = sum over row-r_to columns of C^l[(i, r_from), (., r_to)] p."""
        nx = self.nx
        C = self.layers[l]["C"]
        blk = C[r_from * nx:(r_from + 1) * nx, r_to * nx:(r_to + 1) * nx]
        return blk @ p

    def local_rhs(self, l: int, g: np.ndarray) -> np.ndarray:
        """g^l = chi_{Omega^l} g on the extended strip (eq. local_discrete_sparse_pde)."""
        b = np.zeros((self.q, self.nx), dtype=np.complex128)
        b[self.E:self.E + self.t] = g[l * self.t:(l + 1) * self.t]
        return b

    def solve_local(self, l: int, b: np.ndarray) -> np.ndarray:
        """w^l = (C^l)^{-1} b (local solve, by the banded LU of the x-slow reordering)."""
        lay = self.layers[l]
        perm = lay["perm"]
        x = np.empty(self.q * self.nx, dtype=np.complex128)
        x[perm] = lay["lu"].solve(np.ascontiguousarray(b).ravel()[perm])
        return x.reshape(self.q, self.nx)

    def inject_from_above(self, l: int, b: np.ndarray, w_up: np.ndarray) -> None:
        """b += -delta_n C^l_{n,n+1} w^{l+1}_1 + delta_{n+1} C^l_{n+1,n} w^{l+1}_0 (eq. pde_GRF_down)."""
        E, t = self.E, self.t
        rn = E + t - 1
        b[rn] -= self.coupling(l, rn, rn + 1, w_up[E])       # w^{l+1}_1
        b[rn + 1] += self.coupling(l, rn + 1, rn, w_up[E - 1])  # w^{l+1}_0

    def inject_from_below(self, l: int, b: np.ndarray, v_dn: np.ndarray, w_self: np.ndarray) -> None:
        """b += -delta_1 C^l_{1,0} p_0 + delta_0 C^l_{0,1} p_1 with the up-going traces
        p_0 = v^{l-1}_n - w^l_0, p_1 = v^{l-1}_{n+1} (upward sweep; reading in the module docstring)."""
        E, t = self.E, self.t
        b[E] -= self.coupling(l, E, E - 1, v_dn[E + t - 1] - w_self[E - 1])   # p_0
        b[E - 1] += self.coupling(l, E - 1, E, v_dn[E + t])                    # p_1 = v^{l-1}_{n+1}


def sweep(lay: Layering, g: np.ndarray) -> np.ndarray:
    """Algorithm 1 (Gauss-Seidel preconditioner, Sec. 3.4) on horizontal layers."""
    L, E, t = lay.L, lay.E, lay.t
    gl = [None] * L
    w = [None] * L
    for l in range(L - 1, -1, -1):          # downwards sweep
        gl[l] = lay.local_rhs(l, g)
        if l != L - 1:
            lay.inject_from_above(l, gl[l], w[l + 1])
        w[l] = lay.solve_local(l, gl[l])
    v = [None] * L
    for l in range(L):                      # upwards sweep
        if l != 0:
            lay.inject_from_below(l, gl[l], v[l - 1], w[l])
        v[l] = lay.solve_local(l, gl[l])
    out = np.empty_like(g, dtype=np.complex128)
    for l in range(L):                      # concatenation
        out[l * t:(l + 1) * t] = v[l][E:E + t]
    return out


class BiDirectional:
    """Algorithm 2 (bi-directional preconditioner, Sec. 3.5).

    Holds the horizontal layering of C and the horizontal layering of the
    transposed grid (vertical layers of the original one).
    """

    def __init__(self, m: np.ndarray, st: sparsify.Stencils, omega: float, L: int,
                 E: int = 10, shift: float = 10.0):
        self.m, self.st, self.omega = m, st, omega
        self.C = sparsify.matrix_C(m, st, omega)
        self.horizontal = Layering(m, st, omega, L, E, shift)
        self.vertical = Layering(m.T.copy(), st.transposed(), omega, L, E, shift)

    def precond_horizontal(self, g):
        return sweep(self.horizontal, g)

    def precond_vertical(self, g):
        return sweep(self.vertical, g.T.copy()).T.copy()

    def __call__(self, g: np.ndarray) -> np.ndarray:
        u1 = self.precond_horizontal(g)                       # up-down pass
        e = g - (self.C @ u1.ravel()).reshape(g.shape)        # iterative refinement
        u2 = self.precond_vertical(e)                         # left-right pass
        return u1 + u2
