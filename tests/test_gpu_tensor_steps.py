"""Block-cyclic-reduction steps on the tensor cores (mixed precision) through the C ABI.

The local solves (C^l)^{-1} b of Algorithm 1 (Sec. 3.4; factors of Sec. 4.1) run their
reduction steps as TF32 matrix products (tcgen05.mma, factor tiles by TMA).  Checks:
  * every strip height class (q = 24, 36, 84, 104: 1 to 4 swizzle atoms of K per
    plane) and both directions against the oracle's banded-LU local solve, with a
    bound from TF32 rounding (2^-11 relative per operand) and the CUDA-core FP32
    form as the control;
  * a batch of up to 32 right-hand sides gives each member what a batch of one gives
    (the products of different members never mix);
  * both with the reduction steps of every level and with the levels at and above the
    first one of at most 32 blocks replaced by one product with the precomputed inverse of
    that level's reduced system (both round to TF32; the two agree to that rounding);
  * Algorithm 2 and the inner solve stay usable as a preconditioner: the solve
    converges to the oracle's solution (the FP64 residual judges);
  * no step ran out of its bounded waits.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import polarized, solver as osolver, sparsify  # noqa: E402
from paper_1602_07652_gb300 import binding, inputs  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    binding.load()


# (n, L, E) -> q = n / L + 2E: 24 (1 atom of 32), 36 (2), 84 (3), 104 (4)
QCASES = [(48, 3, 4), (64, 4, 10), (256, 4, 10), (192, 2, 4)]


@pytest.mark.parametrize("dense", [1, 0])
@pytest.mark.parametrize("n,L,E", QCASES)
def test_tensor_core_local_solves_match_oracle(n, L, E, dense):
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=n + L)
    before = binding.device_timeouts()   # cumulative since the library was loaded
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_reduced_inverse(dense)
    st = sparsify.Stencils(n, 1.0 / n, w)
    lays = (polarized.Layering(m, st, w, L, E), polarized.Layering(m.T.copy(), st.transposed(), w, L, E))
    worst_tc, worst_cc = 0.0, 0.0
    for d in (0, 1):
        for l in sorted({0, L // 2, L - 1}):
            b = inputs.random_field(n, 300 + 7 * l + d, nz=lays[d].q)
            ref = lays[d].solve_local(l, b)
            s.ls_set_tensor_steps(2)   # always (one right-hand side)
            x_tc = s.ls_local_solve(d, l, cuda(b)).cpu().numpy()
            s.ls_set_tensor_steps(0)
            x_cc = s.ls_local_solve(d, l, cuda(b)).cpu().numpy()
            worst_tc = max(worst_tc, rel(x_tc, ref))
            worst_cc = max(worst_cc, rel(x_cc, ref))
    print("n=%d L=%d E=%d q=%d reduced inverse %d: TF32 tensor-core local solve rel err %.2e, FP32 CUDA cores %.2e"
          % (n, L, E, lays[0].q, dense, worst_tc, worst_cc))
    assert worst_cc < 2e-4
    assert worst_tc < 3e-2
    assert binding.device_timeouts() == before
    s.close()


@pytest.mark.parametrize("dense", [1, 0])
@pytest.mark.parametrize("nb", [5, 12, 32])
def test_tensor_core_batch_members_are_independent(nb, dense):
    # NB templates 8, 16, 32; member b of a batch = the same field alone
    n, L, E = 128, 2, 10
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=31)
    before = binding.device_timeouts()
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_tensor_steps(2)
    s.ls_set_reduced_inverse(dense)
    g = torch.stack([cuda(inputs.random_field(n, 500 + b)) for b in range(nb)]).contiguous()
    v = s.ls_precond_bd_batch(g)
    for b in sorted({0, nb // 2, nb - 1}):
        vb = s.ls_precond_bd(g[b].contiguous())
        assert torch.equal(v[b], vb) or rel(v[b].cpu(), vb.cpu()) < 1e-6, b
    assert binding.device_timeouts() == before
    s.close()


def test_reduced_inverse_and_level_steps_agree():
    # one Algorithm 2 application at 256^2 (levels: 256, 128, 64, 32 blocks -> the inverse
    # of level 3's 32-block system, 2688 unknowns) with and without the reduced inverse
    n, L, E = 256, 4, 10
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=77)
    before = binding.device_timeouts()
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_tensor_steps(2)
    g = torch.stack([cuda(inputs.random_field(n, 900 + b)) for b in range(16)]).contiguous()
    s.ls_set_reduced_inverse(1)
    v1 = s.ls_precond_bd_batch(g).clone()
    v1b = s.ls_precond_bd_batch(g).clone()
    s.ls_set_reduced_inverse(0)
    v0 = s.ls_precond_bd_batch(g).clone()
    d = rel(v1.cpu(), v0.cpu())
    print("reduced inverse vs level steps: rel diff %.2e" % d)
    assert torch.equal(v1, v1b)   # fixed summation order: reproducible
    assert d < 1e-2               # both within the TF32 error (about 1e-3) of the exact solve
    assert binding.device_timeouts() == before
    with pytest.raises(binding.LSError) as e:
        s.ls_set_reduced_inverse(2)
    assert e.value.code == -1
    s.close()


def test_tensor_core_preconditioner_solve_matches_oracle():
    n, L, E = 128, 2, 10
    w = inputs.omega_for_ppw(n, 10.24)
    m = inputs.bump_medium(n, nbumps=10, seed=41)
    th = inputs.seeded_angle(5)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    out = {}
    for tc in (2, 0):
        s.ls_set_tensor_steps(tc)
        u, st = s.ls_solve_plane_wave(th, 1e-10)
        out[tc] = (u.cpu().numpy(), st)
    s.ls_set_tensor_steps(2)
    s.ls_set_reduced_inverse(0)
    u, st = s.ls_solve_plane_wave(th, 1e-10)
    out[3] = (u.cpu().numpy(), st)
    prob = osolver.Problem(m, w, L=L, E=E)
    u_ref, _ = osolver.solve(prob, prob.rhs(th), tol=1e-12)
    e1, e0 = rel(out[2][0], u_ref), rel(out[0][0], u_ref)
    print("solve: tensor cores rel err %.2e (outer %d, inner %d); CUDA cores %.2e (outer %d, inner %d)"
          % (e1, out[2][1]["outer_iters"], out[2][1]["inner_iters_total"], e0, out[0][1]["outer_iters"],
             out[0][1]["inner_iters_total"]))
    e3 = rel(out[3][0], u_ref)
    print("solve: tensor cores without the reduced inverse rel err %.2e (outer %d)" % (e3, out[3][1]["outer_iters"]))
    assert e1 < 1e-6 and e0 < 1e-6 and e3 < 1e-6
    assert out[2][1]["true_rel_residual"] <= 1e-10
    s.close()


def test_tensor_steps_switch_needs_the_mixed_factors():
    n = 32
    s = binding.Solver(cuda(inputs.gaussian_disk_medium(n)), 2 * math.pi * 4, layers=2, ext=4)
    s.ls_factor()   # FP64: no tensor-core form
    for on in (1, 2):
        with pytest.raises(binding.LSError) as e:
            s.ls_set_tensor_steps(on)
        assert e.value.code == -8   # LS_ESTATE
    s.ls_set_tensor_steps(0)
    with pytest.raises(binding.LSError) as e:
        s.ls_set_tensor_steps(3)
    assert e.value.code == -1
    s.close()
