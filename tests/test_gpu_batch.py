"""Batched right-hand sides through the C ABI (GPU).

A batch shares H (one scatterer, many incident directions, Sec. 5) and must
give, member by member, what the one-at-a-time entry points give:
  * Algorithm 2 on a block of fields equals Algorithm 2 on each field;
  * the lockstep batched solve reaches the tolerance on every member and its
    fields match the single solves (the same iterates up to rounding), and the
    oracle's solution on the small case;
  * degenerate members (f_b = 0) and bad input (NaN) behave as in ls_solve.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import solver as osolver  # noqa: E402
from paper_1602_07652_gb300 import binding, inputs  # noqa: E402


def rel(a, b):
    return float(torch.linalg.norm((a - b).flatten()) / torch.linalg.norm(b.flatten()))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    binding.load()


def _fields(n, nb, seed):
    return torch.stack([cuda(inputs.random_field(n, seed + b)) for b in range(nb)]).contiguous()


@pytest.mark.parametrize("prec,nb", [(binding.LS_FP64, 1), (binding.LS_FP64, 3), (binding.LS_FP64, 4),
                                     (binding.LS_MIXED, 2), (binding.LS_MIXED, 5), (binding.LS_MIXED, 8)])
def test_batched_bd_equals_per_member_bd(prec, nb):
    # ragged: 96 = 6 layers of 16 rows, q = 24 (one warp of rows); nb not a power of two
    n, L, E = 96, 6, 4
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=5)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    if prec == binding.LS_MIXED:
        s.ls_set_tensor_steps(0)   # the CUDA-core steps (the tensor-core form: test_gpu_tensor_steps)
    g = _fields(n, nb, 100)
    v = s.ls_precond_bd_batch(g)
    torch.cuda.synchronize()
    for b in range(nb):
        vb = s.ls_precond_bd(g[b].contiguous())
        err = rel(v[b], vb)
        assert err < (1e-13 if prec == binding.LS_FP64 else 1e-6), (b, err)
    s.close()


@pytest.mark.parametrize("prec", [binding.LS_FP64, binding.LS_MIXED])
def test_batched_bd_with_two_warps_of_rows(prec):
    # q = 2 * 8 + 32 = 48 > 32 rows: two rows per lane in the block mat-vecs
    n, L, E = 128, 4, 8
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.gaussian_disk_medium(n)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    nb = 4
    g = _fields(n, nb, 7)
    v = s.ls_precond_bd_batch(g)
    for b in range(nb):
        assert rel(v[b], s.ls_precond_bd(g[b].contiguous())) < (1e-13 if prec == binding.LS_FP64 else 1e-6)
    s.close()


def test_batched_bd_rejects_oversized_batches():
    n = 32
    s64 = binding.Solver(cuda(inputs.gaussian_disk_medium(n)), 2 * math.pi * 4, layers=2, ext=4)
    s64.ls_factor()
    with pytest.raises(binding.LSError) as e:
        s64.ls_precond_bd_batch(_fields(n, 5, 0))  # FP64 takes at most 4
    assert e.value.code == -1
    s64.close()
    smx = binding.Solver(cuda(inputs.gaussian_disk_medium(n)), 2 * math.pi * 4, layers=2, ext=4,
                         precision=binding.LS_MIXED)
    smx.ls_factor()
    with pytest.raises(binding.LSError) as e:
        smx.ls_precond_bd_batch(_fields(n, binding.LS_MAX_BD_BATCH + 1, 0))
    assert e.value.code == -1
    smx.ls_set_tensor_steps(0)   # the CUDA-core steps take at most 8
    with pytest.raises(binding.LSError) as e:
        smx.ls_precond_bd_batch(_fields(n, 9, 0))
    assert e.value.code == -1
    smx.close()


@pytest.mark.parametrize("prec", [binding.LS_FP64, binding.LS_MIXED])
def test_batched_solve_matches_single_solves_and_oracle(prec):
    n, L, E = 64, 4, 8
    w = 2 * math.pi * 8
    m = inputs.bump_medium(n, nbumps=6, seed=21)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    if prec == binding.LS_MIXED:
        s.ls_set_tensor_steps(2)   # one form for the batch and the single solves
    thetas = [0.0, 0.7, 2.1, 4.4, 5.9]
    f = torch.stack([s.ls_incident_rhs(t) for t in thetas]).contiguous()
    tol = 1e-10
    u, st, rc = s.ls_solve_batch(f, tol)
    assert rc == 0
    assert st["true_rel_residual"] <= tol
    outer = 0
    for b, t in enumerate(thetas):
        ub, stb, _ = s.ls_solve(f[b].contiguous(), tol)
        outer += stb["outer_iters"]
        assert rel(u[b], ub) < 1e-9, (b, rel(u[b], ub))
    assert st["outer_iters"] == outer  # the same iterates, member by member
    prob = osolver.Problem(m, w, L=L, E=E)
    for b in (0, 3):
        u_ref, _ = osolver.solve(prob, prob.rhs(thetas[b]), tol=1e-12)
        assert rel(u[b].cpu(), torch.from_numpy(u_ref)) < 1e-6
    s.close()


def test_packed_members_match_unpacked_batch():
    # Algorithm 2 on the members still iterating only (packed into the leading slots)
    # versus on the whole batch up to the last member still iterating: the same
    # converged fields, fewer fields through Algorithm 2.
    n, L, E = 96, 4, 6
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=10, seed=5)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    thetas = [0.3 * k + 0.1 for k in range(12)]
    f = torch.stack([s.ls_incident_rhs(t) for t in thetas]).contiguous()
    tol = 1e-9
    s.ls_set_pack_members(0)
    u0, st0, rc0 = s.ls_solve_batch(f, tol)
    h0 = s.ls_get_sweep_histogram()
    s.ls_set_pack_members(1)
    u1, st1, rc1 = s.ls_solve_batch(f, tol)
    h1 = s.ls_get_sweep_histogram()
    # the histogram of batch sizes accounts for every field through Algorithm 2
    assert sum(k * v for k, v in h0.items()) == st0["sweep_fields"]
    assert sum(k * v for k, v in h1.items()) == st1["sweep_fields"]
    assert rc0 == 0 and rc1 == 0
    assert st0["true_rel_residual"] <= tol and st1["true_rel_residual"] <= tol
    print("fields through Algorithm 2: unpacked %d packed %d; outer %d / %d" % (
        st0["sweep_fields"], st1["sweep_fields"], st0["outer_iters"], st1["outer_iters"]))
    assert st1["sweep_fields"] <= st0["sweep_fields"]
    for b in range(len(thetas)):
        assert rel(u1[b], u0[b]) < 1e-7, (b, rel(u1[b], u0[b]))
    with pytest.raises(binding.LSError):
        s.ls_set_pack_members(3)
    s.close()


def test_batched_solve_with_a_zero_member_and_ragged_size():
    n, L, E = 48, 3, 4
    w = inputs.omega_for_ppw(n, 8.0)
    m = inputs.bump_medium(n, nbumps=8, seed=11)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    f = torch.stack([s.ls_incident_rhs(0.4), torch.zeros((n, n), dtype=torch.complex128, device="cuda"),
                     s.ls_incident_rhs(3.0)]).contiguous()
    u = torch.full_like(f, 5.0)
    u, st, rc = s.ls_solve_batch(f, 1e-8, u)
    assert rc == 0
    assert not u[1].abs().max().item()
    for b in (0, 2):
        ub, _, _ = s.ls_solve(f[b].contiguous(), 1e-8)
        assert rel(u[b], ub) < 1e-7
    s.close()


def test_batched_solve_rejects_nan_and_bad_counts():
    n = 32
    s = binding.Solver(cuda(inputs.gaussian_disk_medium(n)), 2 * math.pi * 4, layers=2, ext=4)
    s.ls_factor()
    f = torch.stack([s.ls_incident_rhs(0.0), s.ls_incident_rhs(1.0)]).contiguous()
    f[1, 3, 3] = float("nan")
    _, _, rc = s.ls_solve_batch(f, 1e-8, check=False)
    assert rc == -6
    u = torch.empty_like(f)
    lib = binding.load()
    rc = lib.ls_solve_batch(s._h, 0, binding._ptr(f), 1e-8, binding._ptr(u), 0, None)
    assert rc == -1
    rc = lib.ls_solve_batch(s._h, binding.LS_MAX_BATCH + 1, binding._ptr(f), 1e-8, binding._ptr(u), 0, None)
    assert rc == -1
    s.close()


def test_group_of_uneven_problems_matches_one_by_one_solves():
    # independent problems of different sizes and media, each on its own stream
    sizes = [(48, 3, 4), (64, 4, 6), (96, 6, 4), (128, 4, 8), (64, 2, 10)]
    solvers, fs = [], []
    for k, (n, L, E) in enumerate(sizes):
        w = inputs.omega_for_ppw(n, 10.0)
        m = inputs.bump_medium(n, nbumps=6, seed=40 + k)
        st = torch.cuda.Stream()
        prec = binding.LS_MIXED if k % 2 else binding.LS_FP64
        s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec, stream=st)
        s.ls_factor()
        solvers.append(s)
        fs.append(s.ls_incident_rhs(0.3 * k))
    torch.cuda.synchronize()
    us, stats, status = binding.solve_group(solvers, fs, 1e-8)
    torch.cuda.synchronize()
    assert status == [0] * len(sizes)
    for s, f, u, st in zip(solvers, fs, us, stats):
        u1, st1, _ = s.ls_solve(f, 1e-8)
        torch.cuda.synchronize()
        assert rel(u, u1) < 1e-12  # same kernels, same reduction order
        assert st["outer_iters"] == st1["outer_iters"]
        assert st["true_rel_residual"] <= 1e-8
    for s in solvers:
        s.close()


def test_group_rejects_a_handle_given_twice():
    n = 32
    s = binding.Solver(cuda(inputs.gaussian_disk_medium(n)), 2 * math.pi * 4, layers=2, ext=4)
    s.ls_factor()
    f = s.ls_incident_rhs(0.0)
    with pytest.raises(binding.LSError) as e:
        binding.solve_group([s, s], [f, f.clone()], 1e-8)
    assert e.value.code == -1
    s.close()


@pytest.mark.parametrize("prec", [binding.LS_FP64, binding.LS_MIXED])
def test_autotuner_choices_keep_results(prec):
    n, L, E = 128, 4, 8
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=3)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    f = torch.stack([s.ls_incident_rhs(t) for t in (0.1, 1.3, 2.9, 4.0)]).contiguous()
    u0, _, _ = s.ls_solve_batch(f, 1e-9)
    y0 = s.ls_apply_mixed(f[0].contiguous())
    t = s.ls_autotune(nrhs=4, reps=2)
    assert t["fft_variant"] in range(9) and t["bd_chunk"] in (1, 2, 4)
    assert all(x > 0 for x in t["fft_ms"])  # P = 256: every tile shape exists
    assert all(x > 0 for x in t["bd_ms_per_rhs"][:3])
    u1, st, rc = s.ls_solve_batch(f, 1e-9)
    assert rc == 0 and st["true_rel_residual"] <= 1e-9
    assert rel(u1, u0) < 1e-7
    assert rel(s.ls_apply_mixed(f[0].contiguous()), y0) < 2e-5
    s.close()


def test_batch_larger_than_a_chunk_runs_two_concurrent_lanes():
    # 12 members in mixed precision: Algorithm 2 in chunks of 8 and 4 on two streams
    n, L, E = 64, 4, 8
    w = 2 * math.pi * 8
    m = inputs.bump_medium(n, nbumps=6, seed=31)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_tensor_steps(0)   # the CUDA-core steps: chunks of at most 8
    thetas = [0.5 * k for k in range(12)]
    f = torch.stack([s.ls_incident_rhs(t) for t in thetas]).contiguous()
    u, st, rc = s.ls_solve_batch(f, 1e-9)
    assert rc == 0 and st["true_rel_residual"] <= 1e-9
    for b in (0, 7, 8, 11):
        ub, _, _ = s.ls_solve(f[b].contiguous(), 1e-9)
        assert rel(u[b], ub) < 1e-9, (b, rel(u[b], ub))
    # and the bare preconditioner on 8 + 4 fields equals its per-field application
    g = _fields(n, 8, 50)
    v8 = s.ls_precond_bd_batch(g)
    for b in (0, 5):
        assert rel(v8[b], s.ls_precond_bd(g[b].contiguous())) < 1e-6
    s.close()



@pytest.mark.parametrize("n,L,E,nb", [(96, 6, 4, 3), (128, 4, 8, 8), (256, 4, 10, 5), (64, 2, 10, 1)])
def test_split_and_unsplit_reduction_steps_agree(n, L, E, nb):
    # q = 24, 48, 84 (the 2048^2 workload's blocks: 64 rows + 2 x 10), 52; both
    # forms of the reduction give Algorithm 2's result to FP32 rounding on every
    # member of a ragged batch, and the split form is reproducible run to run
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=8)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_tensor_steps(0)   # the split / unsplit forms are those of the CUDA-core steps
    g = _fields(n, nb, 300)
    s.ls_set_reduction(0)
    v0 = s.ls_precond_bd_batch(g).clone()
    s.ls_set_reduction(1)
    v1 = s.ls_precond_bd_batch(g).clone()
    assert torch.equal(s.ls_precond_bd_batch(g), v1)
    for b in range(nb):
        assert rel(v1[b], v0[b]) < 1e-6, (b, rel(v1[b], v0[b]))
    assert rel(v1[nb - 1], s.ls_precond_bd(g[nb - 1].contiguous())) < 1e-6
    with pytest.raises(binding.LSError):
        s.ls_set_reduction(2)
    s.close()


def test_unsplit_reduction_inside_a_batched_solve_meets_the_oracle():
    n, L, E = 256, 4, 10
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=9)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_reduction(0)
    thetas = [0.2, 2.5, 4.0]
    f = torch.stack([s.ls_incident_rhs(t) for t in thetas]).contiguous()
    u, st, rc = s.ls_solve_batch(f, 1e-9)
    assert rc == 0 and st["true_rel_residual"] <= 1e-9
    prob = osolver.Problem(m, w, L=L, E=E)
    u_ref, _ = osolver.solve(prob, prob.rhs(thetas[1]), tol=1e-12)
    assert rel(u[1].cpu(), torch.from_numpy(u_ref)) < 1e-7
    s.close()


def test_sixty_four_directions_in_one_call_match_single_solves():
    # the paper's 64 incident waves per medium (Sec. 5) in one ls_solve_batch call:
    # Algorithm 2 runs in chunks of up to 32 on concurrent lanes
    n, L, E = 96, 2, 6
    w = inputs.omega_for_ppw(n, 10.0)
    m = inputs.bump_medium(n, nbumps=6, seed=64)
    s = binding.Solver(cuda(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    s.ls_factor()
    s.ls_set_tensor_steps(2)   # one form for the batch and the single solves
    B = binding.LS_MAX_BATCH
    assert B == 64
    f = torch.stack([s.ls_incident_rhs(2 * math.pi * j / B) for j in range(B)]).contiguous()
    u, st, rc = s.ls_solve_batch(f, 1e-9)
    assert rc == 0 and st["true_rel_residual"] <= 1e-9
    for b in (0, 31, 32, 63):
        ub, _, _ = s.ls_solve(f[b].contiguous(), 1e-9)
        assert rel(u[b], ub) < 1e-7, b
    s.close()
