"""The no-allocation FP32 LS-apply against the handle-based one (GPU).

ls_apply_f32_noalloc serves callers that must not allocate device memory when
they call it (a memory manager that owns the whole device budget, or a loop
that cannot afford the synchronisation an allocation may cause): its scratch
is a fixed device array inside the library.  It must give what ls_apply_f32
gives for the same contrast and spectrum, call after call, also in place
(y = u), leave the device's free memory unchanged from one call to the next,
and refuse sizes beyond its fixed scratch.  This file is collected last on
purpose.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1602_07652_gb300 import binding, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm((a - b).flatten()) / torch.linalg.norm(b.flatten()))


@pytest.mark.parametrize("n,L,E", [(300, 5, 4), (1024, 16, 10)])
def test_no_alloc_apply_matches_handle_apply_on_consecutive_calls(n, L, E):
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    w = inputs.omega_for_ppw(n, 10.24)
    m = inputs.bump_medium(n, nbumps=8, seed=n)
    s = binding.Solver(torch.from_numpy(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    ghat64, P = s.ls_get_spectrum()
    assert P == 1 << math.ceil(math.log2(2 * n - 1))
    ghat32 = ghat64.to(torch.complex64).contiguous()
    m32 = torch.from_numpy(m).to(device="cuda", dtype=torch.float32).contiguous()
    for seed in (1, 2):  # two calls in a row: the shared scratch keeps the previous call's contents
        u = torch.from_numpy(inputs.random_field(n, seed).astype(np.complex64)).cuda()
        y_ref = s.ls_apply_f32(u)
        y, rc = binding.ls_apply_f32_noalloc(n, m32, ghat32, u)
        torch.cuda.synchronize()
        assert rc == 0
        assert rel(y, y_ref) < 2e-5
    s.close()


def test_no_alloc_apply_rejects_sizes_beyond_its_scratch():
    n = 1025
    m32 = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    g = torch.zeros((2049, 2049), dtype=torch.complex64, device="cuda")
    u = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    y = torch.full_like(u, 7.0)
    _, rc = binding.ls_apply_f32_noalloc(n, m32, g, u, y, check=False)
    assert rc == -9  # LS_ETOOBIG
    assert bool((y == 7.0).all())  # nothing was written


def test_no_alloc_apply_in_place_and_without_device_allocation():
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    n, L, E = 512, 8, 10
    w = inputs.omega_for_ppw(n, 10.24)
    m = inputs.bump_medium(n, nbumps=8, seed=5)
    s = binding.Solver(torch.from_numpy(m), w, layers=L, ext=E, precision=binding.LS_MIXED)
    ghat64, _ = s.ls_get_spectrum()
    ghat32 = ghat64.to(torch.complex64).contiguous()
    m32 = torch.from_numpy(m).to(device="cuda", dtype=torch.float32).contiguous()
    us = [torch.from_numpy(inputs.random_field(n, seed).astype(np.complex64)).cuda() for seed in (7, 8, 9)]
    refs = [s.ls_apply_f32(u) for u in us]
    ys = [torch.empty_like(u) for u in us]
    xs = [u.clone() for u in us]  # every tensor exists before the free memory is read
    binding.ls_apply_f32_noalloc(n, m32, ghat32, us[0], ys[0])  # set-up call (the first on this device if run alone)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for u, x, y in zip(us, xs, ys):
        _, rc = binding.ls_apply_f32_noalloc(n, m32, ghat32, x, x)  # in place: y aliases u
        assert rc == 0
        _, rc = binding.ls_apply_f32_noalloc(n, m32, ghat32, u, y)
        assert rc == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0  # the calls after set-up took no device memory
    for x, y, ref in zip(xs, ys, refs):
        assert rel(x, ref) < 2e-5
        assert rel(y, ref) < 2e-5
    s.close()
