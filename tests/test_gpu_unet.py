"""The learned preconditioner step on the GPU against the FP64 oracle network.

The GPU network stores activations, gradients and weights in BF16 and
accumulates in FP32, so it is compared with the oracle at BF16 accuracy:
outputs to a few 1e-2 relative, every layer's gradient by direction
(cosine > 0.97) and size (relative error < 0.25; a cosine of 0.97 is the same
~25 % relative deviation).  The size bound follows from
the arithmetic: a gradient deep in the backward chain has passed through ~12
BF16 roundings of activations and gradients (2^-8 relative each, accumulating
like a random walk to ~3 %), and where an activation is within BF16 rounding of
zero its ReLU mask can differ from the FP64 one, which moves whole terms; the
measured worst layer is ~16 %.  The oracle itself is pinned by brute force and
finite differences in test_oracle_unet.py.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import solver as osolver, unet  # noqa: E402
from paper_1602_07652_gb300 import binding, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_07652_gb300 import build_lib
    build_lib.build()
    binding.load()


def flat_params(p, levels, c0):
    out = []
    for name, _, _ in unet.layer_shapes(levels, c0):
        out.append(p[name + ".w"].ravel())
        out.append(p[name + ".b"].ravel())
    return np.concatenate(out)


def sample(n, seed):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    e = 0.5 * r + 0.3 * np.roll(r, 1, axis=0) + 0.1j * rng.standard_normal((n, n))
    m = inputs.bump_medium(n, nbumps=4, seed=seed)
    return r, e, m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


LEVELS, C0, N = 3, 16, 32


def make_pair(seed=0):
    p = unet.init_params(levels=LEVELS, c0=C0, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * rng.standard_normal(p[k].shape)
    net = binding.Net(levels=LEVELS, c0=C0, max_batch=2, H=N, W=N, train=True)
    assert net.param_count() == sum(v.size for v in p.values())
    net.set_params(torch.from_numpy(flat_params(p, LEVELS, C0)))
    return p, net


def test_forward_matches_oracle_network():
    p, net = make_pair(0)
    r, _, m = sample(N, 3)
    z = net.forward(torch.from_numpy(r[None]).cuda(), torch.from_numpy(m[None]).cuda())[0].cpu().numpy()
    z_ref = unet.apply(p, r, m, levels=LEVELS)
    assert rel(z, z_ref) < 3e-2
    # parameters round-trip in the oracle's layout
    back = net.get_params().numpy()
    assert np.allclose(back, flat_params(p, LEVELS, C0).astype(np.float32))
    net.close()


def test_gradients_match_oracle_network():
    p, net = make_pair(1)
    r, e, m = sample(N, 4)
    loss = net.train_step(torch.from_numpy(r[None]).cuda(), torch.from_numpy(m[None]).cuda(),
                          torch.from_numpy(e[None]).cuda(), lr=0.0)
    g = net.get_grads().numpy()
    x, s = unet.make_input(r, m)
    t = np.stack([e.real / s, e.imag / s])
    loss_ref, g_ref, _ = unet.loss_and_grad(p, x, t, levels=LEVELS)
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    k = 0
    for name, o, c in unet.layer_shapes(LEVELS, C0):
        for part in (".w", ".b"):
            ref = g_ref[name + part].ravel()
            got = g[k:k + ref.size]
            k += ref.size
            cos = float(np.dot(got, ref) / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30))
            assert cos > 0.97, (name + part, cos)
            assert rel(got, ref) < 0.25, (name + part, rel(got, ref))
    assert k == g.size
    net.close()


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned in FP64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = a32.view(np.uint32).astype(np.uint64)
    r = ((b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_storage_model(p, r, m, e, levels):
    """The network as the GPU stores it: the oracle's FP64 layers (unet.conv3x3 and its
    backward, pooling, upsampling) with every stored activation, gradient and weight copy
    rounded to BF16 where the GPU rounds it; sums are exact (FP64), so what is left between
    the two is the GPU's FP32 accumulation order and the BF16 roundings it flips."""
    x, sc = unet.make_input(r, m)
    x = bf16(x)
    W = {k: (bf16(v) if k.endswith(".w") else v) for k, v in p.items()}
    conv = lambda h, name, act: bf16(np.maximum(unet.conv3x3(h, W[name + ".w"], W[name + ".b"]), 0.0)
                                     if act else unet.conv3x3(h, W[name + ".w"], W[name + ".b"]))
    cache, skips, h = {}, [], x
    for l in range(levels):
        if l > 0:
            h = bf16(unet.avgpool2(h))
        for sfx in ("a", "b"):
            name = "enc%d_%s" % (l, sfx)
            cache[name + ".in"] = h
            h = conv(h, name, True)
            cache[name + ".out"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        up = unet.upsample2(h)
        name = "dec%d_up" % l
        cache[name + ".in"] = up
        h = conv(up, name, True)
        cache[name + ".out"] = h
        h = np.concatenate([h, skips[l]], axis=0)
        for sfx in ("a", "b"):
            name = "dec%d_%s" % (l, sfx)
            cache[name + ".in"] = h
            h = conv(h, name, True)
            cache[name + ".out"] = h
    cache["head.in"] = h
    y = conv(h, "head", False)
    t = np.stack([e.real / sc, e.imag / sc])
    d = y - t
    loss = 0.5 * float(np.mean(d * d))
    g = {}

    def back(name, dy, store=True):   # weight grads from BF16 dy and inputs; dx rounded like the GPU's
        dx, g[name + ".w"], g[name + ".b"] = unet.conv3x3_backward(cache[name + ".in"], W[name + ".w"], dy)
        return bf16(dx) if store else dx

    dh = back("head", bf16(d / d.size))
    dskip = [None] * levels
    for l in range(0, levels - 1):
        for sfx in ("b", "a"):
            name = "dec%d_%s" % (l, sfx)
            dh = back(name, dh * (cache[name + ".out"] > 0))
        c = p["dec%d_up.w" % l].shape[0]
        dskip[l] = dh[c:]
        dh = dh[:c]
        name = "dec%d_up" % l
        dh = bf16(unet.upsample2_backward(back(name, dh * (cache[name + ".out"] > 0))))
    for l in range(levels - 1, -1, -1):
        if dskip[l] is not None:
            dh = bf16(dh + dskip[l])
        for sfx in ("b", "a"):
            name = "enc%d_%s" % (l, sfx)
            dh = back(name, dh * (cache[name + ".out"] > 0), store=(l > 0 or sfx == "b"))
        if l > 0:
            dh = unet.avgpool2_backward(dh)
    return loss, g, sc * (y[0] + 1j * y[1])


@pytest.mark.parametrize("tensor_cores", [1, 0])
def test_forward_and_gradients_match_the_bf16_storage_model(tensor_cores):
    # the GPU network against the same network with BF16 storage at the GPU's rounding points
    # (all sums exact): outputs within a few BF16 ulps (2^-8 relative each), every layer's
    # gradient to cos > 0.999 and 2 % relative L2 (FP32 accumulation over K <= 9 x 2c0 x 4
    # terms and the BF16 roundings it flips)
    p, net = make_pair(5)
    net.set_tensor_cores(tensor_cores)
    r, e, m = sample(N, 6)
    z = net.forward(torch.from_numpy(r[None]).cuda(), torch.from_numpy(m[None]).cuda())[0].cpu().numpy()
    loss = net.train_step(torch.from_numpy(r[None]).cuda(), torch.from_numpy(m[None]).cuda(),
                          torch.from_numpy(e[None]).cuda(), lr=0.0)
    gv = net.get_grads().numpy()
    loss_m, g_m, z_m = bf16_storage_model(p, r, m, e, LEVELS)
    print("BF16 model (tensor cores %d): output rel %.2e, loss rel %.2e" % (tensor_cores, rel(z, z_m),
                                                                             abs(loss - loss_m) / loss_m))
    assert rel(z, z_m) < 4e-3
    assert abs(loss - loss_m) < 4e-3 * loss_m
    k, worst = 0, (1.0, 0.0)
    for name, o, c in unet.layer_shapes(LEVELS, C0):
        for part in (".w", ".b"):
            ref = g_m[name + part].ravel()
            got = gv[k:k + ref.size]
            k += ref.size
            cos = float(np.dot(got, ref) / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30))
            worst = (min(worst[0], cos), max(worst[1], rel(got, ref)))
            assert cos > 0.999, (name + part, cos)
            assert rel(got, ref) < 2e-2, (name + part, rel(got, ref))
    print("BF16 model gradients: worst cos %.6f, worst rel %.2e" % worst)
    net.close()


def test_tensor_core_and_wmma_convolutions_agree():
    # both accumulate BF16 products in FP32 and round the output to BF16: they may differ
    # by the ulps their summation orders flip
    _, net = make_pair(7)
    r, _, m = sample(N, 8)
    rt, mt = torch.from_numpy(r[None]).cuda(), torch.from_numpy(m[None]).cuda()
    net.set_tensor_cores(1)
    z1 = net.forward(rt, mt)[0].cpu().numpy()
    net.set_tensor_cores(0)
    z0 = net.forward(rt, mt)[0].cpu().numpy()
    assert rel(z1, z0) < 4e-3
    assert np.abs(z1 - z0).max() < 3e-2 * np.abs(z0).max()
    net.close()


def test_training_steps_reduce_the_loss_and_batches_are_independent():
    _, net = make_pair(2)
    rs, es, ms = zip(*(sample(N, 10 + b) for b in range(2)))
    r = torch.from_numpy(np.stack(rs)).cuda()
    e = torch.from_numpy(np.stack(es)).cuda()
    m = torch.from_numpy(np.stack(ms)).cuda()
    z2 = net.forward(r, m)
    for b in range(2):
        z1 = net.forward(r[b:b + 1].contiguous(), m[b:b + 1].contiguous())
        assert torch.allclose(z1[0], z2[b])  # same kernels on each sample
    losses = [net.train_step(r, m, e, lr=2e-3) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0], losses[::8]
    net.close()


def test_bad_shapes_are_refused():
    net = binding.Net(levels=LEVELS, c0=C0, max_batch=1, H=N, W=N, train=False)
    r = torch.zeros((1, 48, 48), dtype=torch.complex128, device="cuda")
    m = torch.zeros((1, 48, 48), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LSError) as e:
        net.forward(r, m)   # 48 is not a multiple of 32
    assert e.value.code == -1
    r = torch.zeros((2, 32, 32), dtype=torch.complex128, device="cuda")
    m = torch.zeros((2, 32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LSError) as e:
        net.forward(r, m)   # beyond max_batch * H * W
    assert e.value.code == -9
    with pytest.raises(binding.LSError):
        net.train_step(r[:1].contiguous(), m[:1].contiguous(), r[:1].contiguous(), 1e-3)  # created for inference
    net.close()


@pytest.mark.parametrize("prec", [binding.LS_FP64, binding.LS_MIXED])
def test_solve_with_the_learned_step_still_meets_the_oracle(prec):
    # even an untrained network cannot spoil the solve: FGMRES keeps the plain
    # directions and the FP64 residual decides convergence
    n, L, E = 64, 4, 8
    w = 2 * math.pi * 8
    m = inputs.bump_medium(n, nbumps=6, seed=21)
    s = binding.Solver(torch.from_numpy(m).cuda(), w, layers=L, ext=E, precision=prec)
    s.ls_factor()
    net = binding.Net(levels=3, c0=16, max_batch=1, H=n, W=n, train=False, seed=5)
    s.ls_set_learned(net)
    f = s.ls_incident_rhs(0.4)
    u, st, rc = s.ls_solve(f, 1e-10)
    assert rc == 0 and st["true_rel_residual"] <= 1e-10
    assert st["learned_steps"] >= 1
    prob = osolver.Problem(m, w, L=L, E=E)
    u_ref, _ = osolver.solve(prob, prob.rhs(0.4), tol=1e-12)
    assert rel(u.cpu().numpy(), u_ref) < 1e-6
    s.ls_set_learned(None)
    _, st2, _ = s.ls_solve(f, 1e-10)
    assert st2["learned_steps"] == 0
    s.close()
    net.close()


def test_training_on_solver_pairs_improves_the_learned_correction():
    # what training gains: the predicted correction on held-out media gets closer
    # to the true one, and the solve with the learned step still converges
    from paper_1602_07652_gb300 import learned
    n = 128
    train_data = learned.make_dataset(n, seeds=range(1000, 1012))
    held_out = learned.make_dataset(n, seeds=range(2000, 2003))
    net = binding.Net(levels=4, c0=32, max_batch=4, H=n, W=n, train=True, seed=1)
    before = learned.correction_error(net, held_out)
    losses = learned.train(net, train_data, steps=300, batch=4, lr=1e-3, seed=0)
    after = learned.correction_error(net, held_out)
    cmp = learned.compare_solves(net, n, seeds=[2000], thetas=(0.3,))
    print("held-out correction error %.3f -> %.3f; loss %.3e -> %.3e; outer iterations plain %.1f learned %.1f"
          % (before, after, losses[0], losses[-1], cmp["plain"]["outer"], cmp["learned"]["outer"]))
    assert after < 0.8 * before
    assert losses[-1] < losses[0]
    assert cmp["learned"]["learned_steps"] >= 1
    net.close()
