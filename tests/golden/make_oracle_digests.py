"""Write tests/golden/oracle_digest_<n>.json: digests (digest.py) of the FP64 oracle's
solutions of the full-size problems, for the GPU tests and the benchmark's error report.

Runs the oracle only (oracle.solver: the two-level solve of Sec. 4).  Problems: the
seeded 20-bump medium (seed 0, bumps in the disk r <= 0.4), 10.24 points per
wavelength, layers of 64 rows extended by 10, one plane wave at the seeded angle 0:
  n = 1024: w = 2 pi 100, 16 layers;   n = 2048: w = 2 pi 200, 32 layers.
The oracle first solves to 1e-6 (its iteration counts and time at the benchmark's
tolerance are recorded), then continues the same iteration to 1e-10; the digest is of
that field.  Usage: python tests/golden/make_oracle_digests.py [n ...]  (default 1024 2048)
"""
import json
import math
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import solver  # noqa: E402
from paper_1602_07652_gb300 import inputs  # noqa: E402
from tests.golden import digest  # noqa: E402

TOL, TIGHT = 1e-6, 1e-10


def run(n):
    w = 2 * math.pi * 200 * n / 2048
    L = n // 64
    m = inputs.bump_medium(n, nbumps=20, seed=0)
    theta = inputs.seeded_angle(0)
    t0 = time.perf_counter()
    prob = solver.Problem(m, w, L=L, E=10)
    t1 = time.perf_counter()
    f = prob.rhs(theta)
    u, info = solver.solve(prob, f, tol=TOL)
    t2 = time.perf_counter()
    u2, info2 = solver.solve(prob, f, tol=TIGHT, x0=u)
    t3 = time.perf_counter()
    d = digest.make(u2)
    d.update({"omega": w, "layers": L, "ext": 10, "theta": theta, "medium": "bump_medium(n, 20 bumps, seed 0)",
              "tol": TIGHT, "relres": info2["relres"],
              "at_tol_1e-6": {"outer": info["iters"], "inner_total": int(sum(info["inner_iters"])),
                              "inner_per_outer": info["inner_iters"], "relres": info["relres"],
                              "solve_s": t2 - t1},
              "setup_s": t1 - t0, "continue_s": t3 - t2, "host": platform.machine()})
    return d


if __name__ == "__main__":
    for n in [int(a) for a in sys.argv[1:]] or [1024, 2048]:
        d = run(n)
        path = os.path.join(HERE, "oracle_digest_%d.json" % n)
        with open(path, "w") as fh:
            json.dump(d, fh)
            fh.write("\n")
        print(n, {k: v for k, v in d.items() if k not in ("sketch", "points", "values")}, flush=True)
