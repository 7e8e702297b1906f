"""Oracle solves at the benchmark configurations' full sizes, run in worker processes.

A full-size oracle solve takes tens of seconds on one host core, so the full-size parity tests
start these in a process pool (spawned, so the workers share nothing with the process that
drives the GPU) and collect the results when they need them.  This module imports neither torch
nor the CUDA library.
"""
from __future__ import annotations

import time


def matrix(config: str):
    import workloads as w

    if config == "c2":
        return w.c2_matrix(128)
    if config == "c3":
        return w.c3_matrix(100)
    raise ValueError(config)


def solve(config: str, degree: int, tol: float = 1e-8, m: int = 50, maxit: int = 5000) -> dict:
    """The oracle's PP-GMRES(m) on the configuration's matrix and seeded b, polynomial of the given
    degree from the seeded v0 (the oracle's own construction)."""
    import oracle
    import workloads as w

    a = matrix(config)
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    t0 = time.perf_counter()
    p = oracle.poly_gmres(a, v0, degree)
    r = oracle.gmres(a, b, p, tol=tol, m=m, maxit=maxit)
    return {"x": r.x, "iters": r.iters, "converged": r.converged, "relres": r.relres,
            "seconds": time.perf_counter() - t0}
