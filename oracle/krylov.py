"""Oracle: restarted flexible GMRES (textbook, FP64).

Test infrastructure only (see oracle/__init__.py).

Both levels of the method are Krylov iterations (Sec. 4): the inner level runs
GMRES on C u = A f preconditioned by Algorithm 2 (Algorithm 3), the outer level
GMRES on H u = f preconditioned by Algorithm 3.  Because the inner solve stops
at a tolerance, the outer preconditioner is not a fixed linear map; Sec. 6 names
flexible GMRES as the natural choice, so both levels use the flexible form
(right preconditioning, preconditioned directions Z stored).  With a fixed
linear preconditioner it reduces to right-preconditioned GMRES.

Arnoldi uses modified Gram-Schmidt; the least-squares problem is updated with
Givens rotations; convergence is on the relative residual ||b - A x|| / ||b||,
which is re-checked from the true residual at the end of every cycle.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, b, apply_M=None, tol=1e-6, restart=30, maxit=1000, x0=None):
    """Solve A x = b.  Returns (x, info) with info = dict(iters, relres, converged, history)."""
    b = np.asarray(b, dtype=np.complex128)
    shape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else np.asarray(x0, dtype=np.complex128).ravel().copy()
    hist = []
    if nb == 0.0:
        return np.zeros(shape, dtype=np.complex128), dict(iters=0, relres=0.0, converged=True, history=hist)
    A = lambda v: np.asarray(apply_A(v.reshape(shape)), dtype=np.complex128).ravel()
    M = (lambda v: v) if apply_M is None else (lambda v: np.asarray(apply_M(v.reshape(shape)), dtype=np.complex128).ravel())
    total = 0
    r = bv - A(x) if x0 is not None else bv.copy()
    beta = np.linalg.norm(r)
    relres = beta / nb
    hist.append(relres)
    while relres > tol and total < maxit:
        V = [r / beta]
        Z = []
        Hm = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        gvec = np.zeros(restart + 1, dtype=np.complex128)
        gvec[0] = beta
        k = 0
        for j in range(restart):
            z = M(V[j])
            w = A(z)
            Z.append(z)
            for i in range(j + 1):                      # modified Gram-Schmidt
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            hnext = np.linalg.norm(w)
            Hm[j + 1, j] = hnext
            for i in range(j):                          # previous rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            a, c = Hm[j, j], Hm[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = abs(a) / den if den > 0 else 1.0
            sn[j] = (a / abs(a)) * np.conj(c) / den if abs(a) > 0 else 1.0
            Hm[j, j] = cs[j] * a + sn[j] * c
            Hm[j + 1, j] = 0.0
            gvec[j + 1] = -np.conj(sn[j]) * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            k = j + 1
            relres = abs(gvec[j + 1]) / nb
            hist.append(relres)
            if relres <= tol or total >= maxit:
                break
            V.append(w / hnext)
        # solve the k x k triangular system and update x
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (gvec[i] - Hm[i, i + 1:k] @ y[i + 1:k]) / Hm[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        r = bv - A(x)
        beta = np.linalg.norm(r)
        relres = beta / nb
        hist.append(relres)
    return x.reshape(shape), dict(iters=total, relres=relres, converged=relres <= tol, history=hist)
