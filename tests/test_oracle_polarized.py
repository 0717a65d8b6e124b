"""Pins of the oracle's layered decomposition and polarized-traces sweeps (Sec. 3), CPU only."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import polarized, sparsify
from paper_1602_07652_gb300 import inputs


def _problem(n=32, L=4, E=4, shift=10.0, ppw=8.0, seed=0):
    h = 1.0 / n
    w = inputs.omega_for_ppw(n, ppw)
    st = sparsify.Stencils(n, h, w)
    m = inputs.bump_medium(n, nbumps=6, seed=seed)
    return n, w, st, m, polarized.Layering(m, st, w, L, E, shift)


def test_compatibility_condition():
    # Sec. 3.1: C^l coincides with C on the rows of Omega^l (and its two halo rows' couplings)
    n, w, st, m, lay = _problem()
    C = sparsify.matrix_C(m, st, w).tocsr()
    for l in range(lay.L):
        Cl = lay.layers[l]["C"].tocsr()
        for r in range(lay.E, lay.E + lay.t):
            z = lay.row_global(l, r)
            row_g = C[z * n:(z + 1) * n].toarray()
            row_l = Cl[r * n:(r + 1) * n].toarray()
            for dz in (-1, 0, 1):
                zz = z + dz
                if 0 <= zz < n:
                    rr = r + dz
                    assert np.max(np.abs(row_g[:, zz * n:(zz + 1) * n] - row_l[:, rr * n:(rr + 1) * n])) < 1e-13


def test_grf_exactness_with_exact_traces():
    # eq. pde_GRF_real: with the traces of the global solution, w^l = chi_{Omega^l} v exactly
    for shift in (0.0, 10.0):
        n, w, st, m, lay = _problem(shift=shift)
        C = sparsify.matrix_C(m, st, w).tocsc()
        g = inputs.random_field(n, 11)
        v = spla.spsolve(C, g.ravel()).reshape(n, n)
        E, t = lay.E, lay.t
        for l in range(lay.L):
            b = lay.local_rhs(l, g)
            z1 = l * t                 # global row of local row 1
            zn = (l + 1) * t - 1       # global row of local row n
            if l < lay.L - 1:
                b[E + t - 1] -= lay.coupling(l, E + t - 1, E + t, v[zn + 1])
                b[E + t] += lay.coupling(l, E + t, E + t - 1, v[zn])
            if l > 0:
                b[E] -= lay.coupling(l, E, E - 1, v[z1 - 1])
                b[E - 1] += lay.coupling(l, E - 1, E, v[z1])
            wl = lay.solve_local(l, b)
            assert np.max(np.abs(wl[E:E + t] - v[z1:zn + 1])) < 1e-10 * np.max(np.abs(v))
            outside = np.concatenate([wl[:E], wl[E + t:]])
            assert np.max(np.abs(outside)) < 1e-10 * np.max(np.abs(v))


def test_single_layer_sweep_is_exact_inverse():
    n, w, st, m, lay = _problem(n=24, L=1, E=3)
    C = sparsify.matrix_C(m, st, w).tocsc()
    g = inputs.random_field(n, 2)
    v = polarized.sweep(lay, g)
    assert np.linalg.norm(C @ v.ravel() - g.ravel()) < 1e-12 * np.linalg.norm(g)


def test_sweep_residual_concentrates_at_interfaces():
    # Sec. 3.5: after Algorithm 1 the residual lives on the rows next to the layer interfaces
    n, w, st, m, lay = _problem(n=32, L=4, E=5)
    C = sparsify.matrix_C(m, st, w)
    g = inputs.random_field(n, 3)
    v = polarized.sweep(lay, g)
    res = np.abs((g.ravel() - C @ v.ravel()).reshape(n, n)).max(axis=1)
    t = lay.t
    iface = set()
    for l in range(1, lay.L):
        iface.update({l * t - 1, l * t})
    far = [z for z in range(n) if z not in iface]
    assert max(res[far]) < 1e-11 * np.abs(g).max()
    assert min(res[sorted(iface)]) > 1e-6 * np.abs(g).max()


def test_bidirectional_preconditioner_structure():
    n = 24
    h = 1.0 / n
    w = inputs.omega_for_ppw(n, 8.0)
    st = sparsify.Stencils(n, h, w)
    m = inputs.bump_medium(n, nbumps=4, seed=5)
    bd = polarized.BiDirectional(m, st, w, L=3, E=3)
    g = inputs.random_field(n, 6)
    u1 = bd.precond_horizontal(g)
    e = g - (bd.C @ u1.ravel()).reshape(n, n)
    u2 = bd.precond_vertical(e)
    assert np.allclose(bd(g), u1 + u2, rtol=0, atol=1e-13 * np.abs(u1).max())
    # the vertical pass is the horizontal pass of the transposed problem
    lay_t = polarized.Layering(m.T.copy(), st.transposed(), w, 3, 3)
    assert np.allclose(u2, polarized.sweep(lay_t, e.T.copy()).T, rtol=0, atol=1e-13 * np.abs(u2).max())
    # with one layer in each direction Algorithm 2 is exact (e = 0, u2 = 0)
    bd1 = polarized.BiDirectional(m, st, w, L=1, E=3)
    v = bd1(g)
    assert np.linalg.norm(bd.C @ v.ravel() - g.ravel()) < 1e-12 * np.linalg.norm(g)


def test_cutoff_profile():
    E = 10
    xs = [polarized.cutoff(d, E) for d in range(0, E + 1)]
    assert xs[0] == 1.0 and xs[1] == 1.0 and abs(xs[E]) < 1e-15
    assert all(xs[i] >= xs[i + 1] for i in range(E))


def test_one_sweep_transmits_a_source_from_any_layer():
    # Sec. 3.4: the down sweep carries down-going waves through every layer and the up sweep
    # the up-going ones, so one application of Algorithm 1 reproduces the field of a point
    # source wherever it sits (up to the local absorbing conditions), not only below it.
    import scipy.sparse.linalg as spla
    n, L, E = 128, 4, 10
    w = inputs.omega_for_ppw(n, 10.24)
    st = sparsify.Stencils(n, 1.0 / n, w)
    for m in (np.zeros((n, n)), inputs.bump_medium(n, nbumps=8, seed=2)):
        C = sparsify.matrix_C(m, st, w).tocsc()
        lay = polarized.Layering(m, st, w, L, E)
        t = lay.t
        for l in range(L):
            g = np.zeros((n, n), complex)
            g[l * t + t // 2, n // 3] = 1.0
            v = spla.spsolve(C, g.ravel()).reshape(n, n)
            u = polarized.sweep(lay, g)
            assert np.linalg.norm(u - v) / np.linalg.norm(v) < 6e-2, l   # literal reading: O(1)


def test_bidirectional_iterations_do_not_grow_with_layers():
    # Table 1 trend: Algorithm 2 needs a few GMRES iterations, independent of L
    from oracle import krylov
    n, E = 128, 10
    w = inputs.omega_for_ppw(n, 10.24)
    m = inputs.bump_medium(n, nbumps=10, seed=3)
    st = sparsify.Stencils(n, 1.0 / n, w)
    C = sparsify.matrix_C(m, st, w)
    g = inputs.random_field(n, 1)
    its = []
    for L in (2, 4, 8):
        bd = polarized.BiDirectional(m, st, w, L, E)
        _, info = krylov.fgmres(lambda x: (C @ x.ravel()).reshape(n, n), g, bd, tol=1e-6, restart=30, maxit=30)
        assert info["converged"]
        its.append(info["iters"])
    assert max(its) <= 5, its
