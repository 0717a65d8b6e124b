"""Oracle computations that tests run in spawned worker processes (no torch, no CUDA)."""


def bump_problem_solution(n, w, L, seed, tol, E=10):
    """The oracle's two-level solve (Sec. 4) of the seeded 20-bump problem: medium seed 0,
    one plane wave at the seeded angle `seed`.  Returns (u, info)."""
    from oracle import solver as osolver
    from paper_1602_07652_gb300 import inputs
    m = inputs.bump_medium(n, nbumps=20, seed=0)
    prob = osolver.Problem(m, w, L=L, E=E)
    u, info = osolver.solve(prob, prob.rhs(inputs.seeded_angle(seed)), tol=tol)
    return u, {"iters": info["iters"], "relres": info["relres"], "inner": info["inner_iters"]}
