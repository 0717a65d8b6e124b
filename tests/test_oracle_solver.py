"""Pins of the oracle's two-level solver (Sec. 4), CPU only.

Brute force (dense solve), physics (Mie series of a disk, smooth-medium
self-convergence at the quadrature order of Sec. 2), and the special cases
m = 0 and L = 1.
"""
import math

import numpy as np
import pytest

from oracle import greens, krylov, solver
from paper_1602_07652_gb300 import inputs

from ._mie import mie_scattered


def test_two_level_solution_matches_dense_solve():
    n = 16
    w = 2 * math.pi * 2
    m = inputs.bump_medium(n, nbumps=5, seed=3)
    prob = solver.Problem(m, w, L=2, E=3)
    f = prob.rhs(1.1)
    tol = 1e-10
    u, info = solver.solve(prob, f, tol=tol)
    assert info["converged"]
    Gd = greens.dense_G(n, 1.0 / n, w)
    H = np.eye(n * n) + w * w * Gd * m.ravel()[None, :]
    ud = np.linalg.solve(H, f.ravel()).reshape(n, n)
    assert np.linalg.norm(u - ud) <= 10 * tol * np.linalg.norm(ud) * 100


def test_c1_configuration_converges():
    # 64 x 64, w = 2 pi 8, Gaussian disk medium, theta = 0, 4 layers, tol 1e-8
    n = 64
    prob = solver.Problem(inputs.gaussian_disk_medium(n), 2 * math.pi * 8, L=4)
    f = prob.rhs(0.0)
    u, info = solver.solve(prob, f, tol=1e-8)
    assert info["converged"]
    assert np.linalg.norm(f - prob.apply_H(u)) <= 1e-8 * np.linalg.norm(f)
    assert info["iters"] <= 8 and max(info["inner_iters"]) <= 15


def test_zero_medium_zero_solution():
    n = 32
    prob = solver.Problem(np.zeros((n, n)), 2 * math.pi * 4, L=2, E=4)
    f = prob.rhs(0.5)
    u, info = solver.solve(prob, f, tol=1e-8)
    assert np.array_equal(u, np.zeros_like(u)) and info["iters"] == 0


def test_single_layer_inner_solve_takes_one_iteration():
    n = 24
    prob = solver.Problem(inputs.bump_medium(n, nbumps=3, seed=1), 2 * math.pi * 3, L=1, E=3)
    g = inputs.random_field(n, 8)
    u, info = solver.inner_solve(prob, g, tol=1e-10)
    assert info["iters"] == 1


def test_mie_series_convergence():
    # scattered field of a constant-contrast disk vs its Bessel/Hankel series
    w, m0, a, th = 2 * math.pi * 2, 0.2, 0.2, 0.3
    errs = []
    for n in (32, 64):
        m = inputs.constant_disk_medium(n, m0, a)
        prob = solver.Problem(m, w, L=max(1, n // 32), E=4)
        u, info = solver.solve(prob, prob.rhs(th), tol=1e-10)
        X, Z = inputs.node_coords(n)
        ue = mie_scattered(X, Z, w, m0, a, th)
        errs.append(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    assert errs[0] < 0.06 and errs[1] < 0.5 * errs[0], errs


@pytest.mark.slow
def test_mie_series_convergence_fine():
    w, m0, a, th = 2 * math.pi * 2, 0.2, 0.2, 0.3
    n = 128
    m = inputs.constant_disk_medium(n, m0, a)
    prob = solver.Problem(m, w, L=4, E=6)
    u, info = solver.solve(prob, prob.rhs(th), tol=1e-10)
    X, Z = inputs.node_coords(n)
    ue = mie_scattered(X, Z, w, m0, a, th)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) < 3e-3


def test_smooth_medium_self_convergence_order():
    # Sec. 2: quadrature of order h^4 log h -> nested-grid differences shrink ~16x per halving
    w, th = 2 * math.pi * 2, 0.3
    us = {}
    for n in (16, 32, 64, 128):
        m = inputs.smooth_medium(n, amp=0.3, width=0.3)
        f = greens.rhs(m, 1.0 / n, w, greens.incident_plane_wave(n, w, th))
        us[n], info = krylov.fgmres(lambda v: greens.apply_H(v, m, 1.0 / n, w), f, tol=1e-13,
                                    restart=100, maxit=1000)
        assert info["converged"]
    sub = lambda u, k: u[k - 1::k, k - 1::k]
    d = [np.linalg.norm(us[16] - sub(us[32], 2)), np.linalg.norm(sub(us[32], 2) - sub(us[64], 4)),
         np.linalg.norm(sub(us[64], 4) - sub(us[128], 8))]
    rates = [math.log2(d[i] / d[i + 1]) for i in range(2)]
    assert min(rates) > 3.5, rates


def test_fgmres_textbook_cases():
    # GMRES on a diagonal system converges in as many steps as distinct eigenvalues
    D = np.repeat(np.array([1.0, 2.0 + 1j, -3.0]), 20)
    b = np.ones(60, complex)
    x, info = krylov.fgmres(lambda v: D * v, b, tol=1e-12, restart=10)
    assert info["iters"] == 3 and np.allclose(x, b / D, atol=1e-11)
    # restarted run on a nonnormal bidiagonal matrix still meets the tolerance
    n = 40
    Amat = np.eye(n) * 2 + np.diag(np.ones(n - 1), -1)
    rhs = np.arange(1, n + 1, dtype=complex)
    x, info = krylov.fgmres(lambda v: Amat @ v, rhs, tol=1e-10, restart=5, maxit=400)
    assert np.linalg.norm(Amat @ x - rhs) <= 1e-10 * np.linalg.norm(rhs)
