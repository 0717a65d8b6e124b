"""GPU parity of the operators (LS-apply, spectrum, stencils, local solves, sweeps) vs the oracle.

Every test runs the CUDA path through the C ABI (binding.Solver) and compares it
element by element with the FP64 oracle on the same seeded inputs.
Tolerances: FP64 arithmetic on both sides -> 1e-11 relative; stencil
coefficients come from a Gram eigenproblem on the GPU and an SVD in the oracle,
which agree to ~1e-10, so everything built from them is compared at 1e-7;
FP32 paths at 2e-5 (single precision FFT of length <= 4096: eps_32 * log2 N * few).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import greens, polarized, sparsify  # noqa: E402
from paper_1602_07652_gb300 import binding, inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def worst_line(a, b):
    """Largest relative L2 error over single rows and single columns: an error confined
    to one tile edge or one ragged box shows here, hidden in the whole-field figure."""
    d = np.asarray(a) - np.asarray(b)
    b = np.asarray(b)
    rows = np.linalg.norm(d, axis=1) / np.linalg.norm(b, axis=1)
    cols = np.linalg.norm(d, axis=0) / np.linalg.norm(b, axis=0)
    return float(max(rows.max(), cols.max()))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    binding.load()


CASES = [(16, 2, 3, 6.0), (48, 3, 4, 8.0), (64, 4, 10, 8.0), (100, 5, 6, 10.0)]


@pytest.mark.parametrize("n,L,E,ppw", CASES)
def test_ls_apply_fp64_matches_oracle(n, L, E, ppw):
    w = inputs.omega_for_ppw(n, ppw)
    m = inputs.bump_medium(n, nbumps=6, seed=n)
    s = binding.Solver(cuda(m), w, layers=L, ext=E)
    u = inputs.random_field(n, n + 1)
    y = s.ls_apply(cuda(u)).cpu().numpy()
    assert rel(y, greens.apply_H(u, m, 1.0 / n, w)) < 1e-11
    # the diagonal weight and the spectral quadrant are the oracle's
    assert abs(s.ls_get_diag_weight() - greens.diagonal_weight(1.0 / n, w)) < 1e-15
    g, P = s.ls_get_spectrum()
    assert P == 1 << math.ceil(math.log2(2 * n - 1))
    ref = greens.spectrum(n, 1.0 / n, w, P)[: P // 2 + 1, : P // 2 + 1]
    assert rel(g.cpu().numpy(), ref) < 1e-11
    # in-place apply (u and y alias)
    ud = cuda(u)
    s.ls_apply(ud, ud)
    assert rel(ud.cpu().numpy(), y) < 1e-15
    s.close()


@pytest.mark.parametrize("n,L,E,ppw", CASES[1:3])
def test_ls_apply_fp32_and_incident_rhs(n, L, E, ppw):
    w = inputs.omega_for_ppw(n, ppw)
    m = inputs.bump_medium(n, nbumps=6, seed=n + 5)
    s = binding.Solver(cuda(m), w, layers=L, ext=E)
    u = inputs.random_field(n, 9)
    y32 = s.ls_apply_f32(cuda(u.astype(np.complex64))).cpu().numpy()
    y_ref = greens.apply_H(u, m, 1.0 / n, w)
    assert rel(y32, y_ref) < 2e-5
    ymx = s.ls_apply_mixed(cuda(u)).cpu().numpy()   # FP64 I/O, FP32 arithmetic
    assert rel(ymx, y_ref) < 2e-5
    th = 0.37
    f = s.ls_incident_rhs(th).cpu().numpy()
    f_ref = greens.rhs(m, 1.0 / n, w, greens.incident_plane_wave(n, w, th))
    assert rel(f, f_ref) < 1e-11
    s.close()


# Double-float arithmetic (hi + lo FP32 pairs, unit roundoff about 2^-48 = 3.6e-15 per
# operation; an FFT's error grows like log2 of its length times that): the apply and the
# incident right-hand side agree with the FP64 path on the same spectrum to 5e-14 relative
# (measured: at most 4.6e-15) at every transform length from 64 to 4096, ragged n
# included, and with the FP64 oracle
# as closely as the FP64 path does (1e-11: the GPU's Green's-function table and the
# oracle's agree to about 1e-12, which the right-hand side, without the identity term of
# H, shows undiluted).
@pytest.mark.parametrize("n,L", [(30, 2), (48, 3), (100, 4), (300, 6), (520, 8), (1100, 11)])
def test_double_float_apply_and_rhs(n, L):
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=n + 3)
    s = binding.Solver(cuda(m), w, layers=L, ext=3, precision=binding.LS_MIXED)
    u = inputs.random_field(n, 6)
    y_ref = greens.apply_H(u, m, 1.0 / n, w)
    ydf = s.ls_apply_double_float(cuda(u)).cpu().numpy()
    y64 = s.ls_apply(cuda(u)).cpu().numpy()
    assert rel(ydf, y_ref) < 1e-11
    assert rel(ydf, y64) < 5e-14
    assert worst_line(ydf, y64) < 5e-13
    ud = cuda(u)                       # in place (u and y alias)
    s.ls_apply_double_float(ud, ud)
    assert torch.equal(ud.cpu(), torch.from_numpy(ydf))
    th = 1.13
    f_ref = greens.rhs(m, 1.0 / n, w, greens.incident_plane_wave(n, w, th))
    fdf = s.ls_incident_rhs(th).cpu().numpy()        # LS_MIXED default: double-float
    s.ls_set_double_float(0)
    f64 = s.ls_incident_rhs(th).cpu().numpy()
    print("n=%d apply: df-oracle %.2e df-fp64 %.2e; rhs: df-oracle %.2e fp64-oracle %.2e df-fp64 %.2e" % (
        n, rel(ydf, y_ref), rel(ydf, y64), rel(fdf, f_ref), rel(f64, f_ref), rel(fdf, f64)))
    assert rel(fdf, f64) < 5e-14
    assert rel(fdf, f_ref) < 1e-11
    assert rel(f64, f_ref) < 1e-11
    with pytest.raises(RuntimeError):
        s.ls_set_double_float(2)
    s.close()


# every length of the radix-16 FP32 path (P = 256 .. 2048), with ragged n (P > 2n - 1)
@pytest.mark.parametrize("n,L", [(100, 4), (129, 3), (200, 4), (300, 6), (520, 8), (1000, 10)])
def test_fp32_apply_every_transform_length(n, L):
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=n + 1)
    s = binding.Solver(cuda(m), w, layers=L, ext=3, precision=binding.LS_MIXED)
    u = inputs.random_field(n, 4)
    y_ref = greens.apply_H(u, m, 1.0 / n, w)
    y32 = s.ls_apply_f32(cuda(u.astype(np.complex64))).cpu().numpy()
    ymx = s.ls_apply_mixed(cuda(u)).cpu().numpy()
    assert rel(y32, y_ref) < 2e-5
    assert rel(ymx, y_ref) < 2e-5
    s.close()


# every column-pass tile shape of the autotuner gives the same LS-apply; n = 1100
# (P = 4096) has a ragged last TMA box of 76 rows, n = 100 (P = 256) 8 tiles per CTA
@pytest.mark.parametrize("n,L", [(100, 4), (300, 6), (1000, 10), (1100, 11)])
def test_fp32_apply_every_tile_shape(n, L):
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=n + 2)
    s = binding.Solver(cuda(m), w, layers=L, ext=3, precision=binding.LS_MIXED)
    u = inputs.random_field(n, 5)
    y_ref = greens.apply_H(u, m, 1.0 / n, w)
    ys = {}
    for v in range(9):
        s.ls_set_shapes(v)
        ys[v] = s.ls_apply_mixed(cuda(u)).cpu().numpy()
        assert rel(ys[v], y_ref) < 2e-5, v
        assert worst_line(ys[v], y_ref) < 1e-4, v
        assert np.abs(ys[v] - y_ref).max() < 1e-4 * np.abs(y_ref).max(), v
    # the TMA shapes move the same tiles: the same arithmetic, bit for bit
    assert np.array_equal(ys[6], ys[2]) and np.array_equal(ys[7], ys[5])
    # shape 8 pairs the two columns in FP32x2 instructions: other FMA contractions
    assert rel(ys[8], ys[6]) < 1e-6
    assert binding.device_timeouts() == 0
    with pytest.raises(binding.LSError):
        s.ls_set_shapes(9)
    s.close()


def test_integer_pipe_conversions_match_the_hardware():
    # doubles spread over and beyond the float range (subnormal results, overflow), exact
    # halfway cases of the rounding, signed zeros, infinities, NaN; floats of every class
    rng = np.random.default_rng(7)
    cnt = 1 << 21
    e = rng.integers(1023 - 160, 1023 + 140, cnt).astype(np.uint64)
    mant = rng.integers(0, 1 << 52, cnt, dtype=np.uint64)
    mant[: cnt // 4] = (mant[: cnt // 4] & ~np.uint64((1 << 29) - 1)) | np.uint64(1 << 28)   # halfway
    sign = rng.integers(0, 2, cnt).astype(np.uint64) << np.uint64(63)
    dbits = sign | (e << np.uint64(52)) | mant
    dbits[:8] = np.array([0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000001, 1,
                          0x47EFFFFFE0000000, 0x47EFFFFFF0000000], dtype=np.uint64)
    fbits = rng.integers(0, 1 << 32, cnt, dtype=np.uint64).astype(np.uint32)
    fbits[:6] = np.array([0, 0x80000000, 1, 0x7FFFFF, 0x7F800000, 0x7FC00001], dtype=np.uint32)
    d = torch.from_numpy(dbits.view(np.float64)).cuda()
    f = torch.from_numpy(fbits.view(np.float32)).cuda()
    assert binding.check_conversions(d, f) == 0


def test_axpby_forms_the_residual_on_the_device():
    n = 48
    w = inputs.omega_for_ppw(n, 8.0)
    m = inputs.bump_medium(n, nbumps=4, seed=3)
    s = binding.Solver(cuda(m), w, layers=3, ext=4)
    f = inputs.random_field(n, 21)
    u = inputs.random_field(n, 22)
    r = s.ls_apply(cuda(u))
    s.ls_axpby(1.0, cuda(f), -1.0, r)        # r = f - H u
    ref = f - greens.apply_H(u, m, 1.0 / n, w)
    assert rel(r.cpu().numpy(), ref) < 1e-11
    x = cuda(u)
    s.ls_axpby(0.5 - 2j, x, 3.0 + 1j, x)     # x and y alias
    assert rel(x.cpu().numpy(), (0.5 - 2j) * u + (3.0 + 1j) * u) < 1e-15
    s.close()


def test_zero_medium_apply_is_identity_and_rhs_zero():
    n = 32
    s = binding.Solver(cuda(np.zeros((n, n))), 2 * math.pi * 4, layers=2, ext=4)
    u = inputs.random_field(n, 1)
    assert np.array_equal(s.ls_apply(cuda(u)).cpu().numpy(), u)
    assert not s.ls_incident_rhs(0.2).abs().max().item()
    s.close()


@pytest.mark.parametrize("n,L,E,ppw", CASES[:3])
def test_stencils_and_C_match_oracle(n, L, E, ppw):
    w = inputs.omega_for_ppw(n, ppw)
    m = inputs.bump_medium(n, nbumps=6, seed=2 * n)
    s = binding.Solver(cuda(m), w, layers=L, ext=E)
    st = sparsify.Stencils(n, 1.0 / n, w)
    A, B = s.ls_get_stencils()
    assert np.max(np.abs(A - st.alpha.reshape(9, 9))) < 1e-8
    assert np.max(np.abs(B - st.beta.reshape(9, 9))) < 1e-8 * np.max(np.abs(st.beta))
    v = inputs.random_field(n, 4)
    assert rel(s.ls_apply_A(cuda(v)).cpu().numpy(), sparsify.apply_A(v, st)) < 1e-7
    assert rel(s.ls_apply_C(cuda(v)).cpu().numpy(), sparsify.apply_C(v, m, st, w)) < 1e-7
    s.close()


@pytest.mark.parametrize("prec,tol", [(binding.LS_FP64, 1e-7), (binding.LS_MIXED, 2e-4)])
@pytest.mark.parametrize("n,L,E,ppw", CASES[1:3])
def test_local_solves_match_oracle(n, L, E, ppw, prec, tol):
    w = inputs.omega_for_ppw(n, ppw)
    m = inputs.bump_medium(n, nbumps=6, seed=3 * n)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    if prec == binding.LS_MIXED:
        s.ls_set_tensor_steps(0)   # the FP32 CUDA-core steps (tensor-core TF32 steps: test_gpu_tensor_steps)
    st = sparsify.Stencils(n, 1.0 / n, w)
    lay = polarized.Layering(m, st, w, L, E)
    lay_t = polarized.Layering(m.T.copy(), st.transposed(), w, L, E)
    for d, ly in ((0, lay), (1, lay_t)):
        for l in range(L):
            b = inputs.random_field(n, 100 + l, nz=lay.q)
            x = s.ls_local_solve(d, l, cuda(b)).cpu().numpy()
            assert rel(x, ly.solve_local(l, b)) < tol, (d, l)
    s.close()


@pytest.mark.parametrize("prec,tol", [(binding.LS_FP64, 1e-7), (binding.LS_MIXED, 2e-4)])
@pytest.mark.parametrize("n,L,E,ppw", CASES[1:3])
def test_sweeps_match_oracle(n, L, E, ppw, prec, tol):
    w = inputs.omega_for_ppw(n, ppw)
    m = inputs.bump_medium(n, nbumps=6, seed=4 * n)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    if prec == binding.LS_MIXED:
        s.ls_set_tensor_steps(0)
    st = sparsify.Stencils(n, 1.0 / n, w)
    bd = polarized.BiDirectional(m, st, w, L, E)
    g = inputs.random_field(n, 21)
    gd = cuda(g)
    assert rel(s.ls_sweep(0, gd).cpu().numpy(), bd.precond_horizontal(g)) < tol
    assert rel(s.ls_sweep(1, gd).cpu().numpy(), bd.precond_vertical(g)) < tol
    assert rel(s.ls_precond_bd(gd).cpu().numpy(), bd(g)) < tol
    s.close()


def test_single_layer_sweep_inverts_C():
    n, E = 40, 3
    w = inputs.omega_for_ppw(n, 8.0)
    m = inputs.bump_medium(n, nbumps=4, seed=7)
    s = binding.Solver(cuda(m), w, layers=1, ext=E)
    s.ls_factor()
    g = cuda(inputs.random_field(n, 5))
    v = s.ls_sweep(0, g)
    r = g - s.ls_apply_C(v)
    assert (torch.linalg.norm(r) / torch.linalg.norm(g)).item() < 1e-11
    _, it = s.ls_inner_solve(g, 1e-10)
    assert it == 1
    s.close()


def test_full_size_fp64_apply_sampled():
    # 1024 x 1024, w = 2 pi 100, 20 bumps: sampled outputs against the direct quadrature sum
    n = 1024
    w = 2 * math.pi * 100
    m = inputs.bump_medium(n, nbumps=20, seed=0)
    s = binding.Solver(cuda(m), w, layers=16, ext=10)
    u = inputs.random_field(n, 0)
    y = s.ls_apply(cuda(u)).cpu().numpy()
    rng = np.random.default_rng(1)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n // 2, n // 3)] + [tuple(rng.integers(0, n, 2)) for _ in range(6)]
    ref = greens.apply_H_points(u, m, 1.0 / n, w, pts)
    got = np.array([y[j, i] for j, i in pts])
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    s.close()


def test_full_size_fp32_apply_sampled():
    n = 2048
    w = 2 * math.pi * 200
    m = inputs.bump_medium(n, nbumps=20, seed=0)
    s = binding.Solver(cuda(m), w, layers=32, ext=10, precision=binding.LS_MIXED)
    u = inputs.random_field(n, 0)
    y = s.ls_apply_f32(cuda(u.astype(np.complex64))).cpu().numpy()
    y64 = s.ls_apply(cuda(u)).cpu().numpy()
    pts = [(0, 0), (n - 1, n - 1), (n - 1, 0), (1023, 1024), (5, 2000)]
    ref = greens.apply_H_points(u, m, 1.0 / n, w, pts)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(np.array([y64[j, i] for j, i in pts]) - ref)) < 1e-10 * scale
    assert np.max(np.abs(np.array([y[j, i] for j, i in pts]) - ref)) < 2e-5 * scale
    assert rel(y, y64) < 2e-5
    s.close()


def test_bd_graph_replay_equals_direct_launches():
    n, L, E = 64, 4, 6
    w = inputs.omega_for_ppw(n, 8.0)
    m = inputs.bump_medium(n, nbumps=6, seed=9)
    g = cuda(inputs.random_field(n, 2))
    outs = []
    for graphs in (0, 1):
        o = binding.default_opts()
        o.use_graphs = graphs
        s = binding.Solver(cuda(m), w, layers=L, ext=E, opts=o)
        s.ls_factor()
        outs.append(s.ls_precond_bd(g).cpu())
        outs.append(s.ls_precond_bd(g).cpu())   # replay twice
        s.close()
    assert torch.equal(outs[0], outs[2]) and torch.equal(outs[2], outs[3]) and torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("shape", [6, 8])
def test_tma_wait_that_runs_out_marks_the_tiles_and_is_counted(shape):
    # the barrier expects 16 bytes more than the boxes bring: every CTA's wait runs
    # out after one second with no copy in flight, writes its tiles as NaN, counts
    # itself and returns; the context stays usable and the next apply is exact again
    n, L = 100, 4   # P = 256: 8 CTAs of 16 tiles
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=7)
    s = binding.Solver(cuda(m), w, layers=L, ext=3, precision=binding.LS_MIXED)
    u = cuda(inputs.random_field(n, 5))
    s.ls_set_shapes(shape)
    y_ref = s.ls_apply_mixed(u).cpu()
    before = binding.device_timeouts()
    with pytest.raises(binding.LSError):
        binding.test_tma_shortfall(8)
    binding.test_tma_shortfall(16)
    try:
        y_bad = s.ls_apply_mixed(u).cpu()
    finally:
        binding.test_tma_shortfall(0)
    assert binding.device_timeouts() - before == 8
    assert torch.isnan(y_bad.real).any()
    y = s.ls_apply_mixed(u).cpu()
    assert torch.equal(y, y_ref)
    assert binding.device_timeouts() - before == 8
    s.close()
