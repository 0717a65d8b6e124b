"""Training driver of the learned preconditioner step (ls_net_* in the C ABI).

Residual -> correction pairs come from the plain solver itself: for a seeded
bump medium and an incident plane wave, the converged field u* (tolerance
1e-8) and cruder iterates u_k (looser tolerances) give
    r_k = f - H u_k   (the residual the outer iteration sees),
    e_k = u* - u_k    (the correction that would remove it),
and the network N is trained so that s N(r_k / s, m) ~ e_k, s = RMS(r_k).
Every step runs in the library's kernels (solves, applies, network forward,
backward and Adam); this module only orchestrates them.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import binding, inputs


def pairs_for_medium(n, seed, tols=(3e-1, 1e-1, 3e-2), ppw=10.24, precision=binding.LS_MIXED):
    """(r, e, m) pairs of one seeded medium, on the device."""
    m = inputs.bump_medium(n, nbumps=20, seed=seed)
    w = 2 * math.pi * n / ppw
    s = binding.Solver(torch.from_numpy(m), w, layers=max(1, n // 64), ext=10, precision=precision)
    s.ls_factor()
    f = s.ls_incident_rhs(inputs.seeded_angle(seed))
    u_star, _, _ = s.ls_solve(f, 1e-8, check=False)
    rs, es = [], []
    for tol in tols:
        uk, _, _ = s.ls_solve(f, tol, check=False)
        r = s.ls_apply(uk)                       # H u_k
        s.ls_axpby(1.0, f, -1.0, r)              # r_k = f - H u_k
        e = u_star.clone()
        s.ls_axpby(-1.0, uk, 1.0, e)             # e_k = u* - u_k
        rs.append(r)
        es.append(e)
    s.close()
    md = torch.from_numpy(m).cuda()
    return torch.stack(rs), torch.stack(es), md.expand(len(tols), n, n).contiguous()


def make_dataset(n, seeds, tols=(3e-1, 1e-1, 3e-2)):
    rs, es, ms = [], [], []
    for sd in seeds:
        r, e, m = pairs_for_medium(n, sd, tols)
        rs.append(r)
        es.append(e)
        ms.append(m)
    return torch.cat(rs), torch.cat(es), torch.cat(ms)


def train(net, data, steps, batch, lr=1e-3, seed=0, log_every=0):
    """Adam steps on random batches of the (r, e, m) pairs; returns the losses."""
    r, e, m = data
    rng = np.random.default_rng(seed)
    losses = []
    for k in range(steps):
        idx = torch.from_numpy(rng.choice(r.shape[0], size=batch, replace=False)).cuda()
        lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))  # cosine decay
        loss = net.train_step(r[idx].contiguous(), m[idx].contiguous(), e[idx].contiguous(), lr_k)
        losses.append(loss)
        if log_every and k % log_every == 0:
            print("step %d loss %.4e" % (k, loss), flush=True)
    return losses


def correction_error(net, data):
    """Mean over pairs of ||e - s N(r/s, m)|| / ||e|| (how well the step predicts the correction)."""
    r, e, m = data
    errs = []
    for i in range(r.shape[0]):
        z = net.forward(r[i:i + 1].contiguous(), m[i:i + 1].contiguous())
        errs.append(float(torch.linalg.norm(e[i] - z[0]) / torch.linalg.norm(e[i])))
    return float(np.mean(errs))


def compare_solves(net, n, seeds, tol=1e-6, precision=binding.LS_MIXED, thetas=(0.0, 1.1, 2.3)):
    """Outer iterations and solve time with and without the learned step (same RHS)."""
    out = {"plain": {"outer": [], "time": []}, "learned": {"outer": [], "time": [], "learned_steps": []}}
    for sd in seeds:
        m = inputs.bump_medium(n, nbumps=20, seed=sd)
        s = binding.Solver(torch.from_numpy(m), 2 * math.pi * n / 10.24, layers=max(1, n // 64), ext=10,
                           precision=precision)
        s.ls_factor()
        for th in thetas:
            f = s.ls_incident_rhs(th)
            for key, attach in (("plain", None), ("learned", net)):
                s.ls_set_learned(attach)
                s.ls_solve(f, tol)  # warm (allocations, graphs)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st, _ = s.ls_solve(f, tol)
                torch.cuda.synchronize()
                out[key]["time"].append(time.perf_counter() - t0)
                out[key]["outer"].append(st["outer_iters"])
                if key == "learned":
                    out[key]["learned_steps"].append(st["learned_steps"])
        s.ls_set_learned(None)
        s.close()
    return {k: {kk: float(np.mean(vv)) for kk, vv in v.items()} for k, v in out.items()}
