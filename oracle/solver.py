"""Oracle: the two-level solver (Sec. 4).

Test infrastructure only (see oracle/__init__.py).  FP64 throughout.

  * Inner level, Algorithm 3 (Lippmann-Schwinger preconditioner):
    u = GMRES(C, A f, Algorithm 2, tol = 1e-3).
  * Outer level: GMRES on H u = f (eq. discrete_Lipmann-Schwinger) preconditioned
    by Algorithm 3; flexible GMRES (Sec. 6) because Algorithm 3 is not a fixed
    linear map.  Convergence on the true relative residual ||f - H u|| / ||f||.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import greens, krylov, polarized, sparsify


@dataclass
class Problem:
    """Discrete problem of Sec. 2 plus the inner-level machinery of Sec. 3."""
    m: np.ndarray
    omega: float
    L: int
    E: int = 10
    shift: float = 10.0
    h: float = field(init=False)
    n: int = field(init=False)

    def __post_init__(self):
        self.n = self.m.shape[0]
        self.h = 1.0 / self.n
        self.st = sparsify.Stencils(self.n, self.h, self.omega)
        self.A = sparsify.matrix_A(self.n, self.st)
        self.bd = polarized.BiDirectional(self.m, self.st, self.omega, self.L, self.E, self.shift)
        self.C = self.bd.C
        # FFT of the circulant embedding of G, computed once (greens.apply_H's arithmetic)
        self.conv = greens.Convolution(self.n, self.h, self.omega)

    def apply_H(self, u):
        return self.conv.H(u, self.m)

    def apply_A(self, r):
        return (self.A @ r.ravel()).reshape(r.shape)

    def apply_C(self, v):
        return (self.C @ v.ravel()).reshape(v.shape)

    def rhs(self, theta: float):
        return self.conv.rhs(self.m, greens.incident_plane_wave(self.n, self.omega, theta))


def inner_solve(prob: Problem, g, tol=1e-3, restart=30, maxit=300):
    """GMRES on C u = g preconditioned by Algorithm 2 (inner level of Algorithm 3)."""
    return krylov.fgmres(prob.apply_C, g, prob.bd, tol=tol, restart=restart, maxit=maxit)


def ls_preconditioner(prob: Problem, f, inner_tol=1e-3, stats=None):
    """Algorithm 3: u = GMRES(C, A f, BiDirectionalPreconditioner, tol = inner_tol)."""
    u, info = inner_solve(prob, prob.apply_A(f), tol=inner_tol)
    if stats is not None:
        stats.append(info["iters"])
    return u


def solve(prob: Problem, f, tol=1e-8, inner_tol=1e-3, restart=50, maxit=500, x0=None):
    """Outer level: flexible GMRES on H u = f preconditioned by Algorithm 3.

    x0: optional starting iterate (e.g. a looser solve continued to a tighter
    tolerance); the tolerance stays relative to ||f||.
    """
    inner = []
    u, info = krylov.fgmres(prob.apply_H, f, lambda v: ls_preconditioner(prob, v, inner_tol, inner),
                            tol=tol, restart=restart, maxit=maxit, x0=x0)
    info["inner_iters"] = inner
    return u, info
