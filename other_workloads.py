"""The configurations other than the benchmark line (run by `bench.py --workload ...`).

c1  2D 64^2 upwind convection-diffusion, Pe 10, degree 10, GMRES(50), float64 (latency-bound)
c3  perturbed 27-point stencil on 100^3, degree 25 in float32 with float64 refinement, error
    against the float64 solve of the same system
c4  256 uneven 2D systems (sides log-uniform 32..448, Pe U[1,100]), degree 15, GMRES(30),
    float32 inner + float64 refinement, one batched launch vs. solving them one by one
c5  adjoint: 3D 64^3 (Pe 50), degree 20; dL/db and dL/dvals of L = ||x - x_t||^2 against central
    differences (h = 1e-6) on 50 sampled entries each

Each prints one JSON line.  Times are CUDA-event times on the solver's stream.
"""
from __future__ import annotations

import json
import os
import statistics
import time

import numpy as np

import workloads as w


def _dev():
    import torch

    return torch.device("cuda", 0)


def _T(a, dt):
    import torch

    return torch.as_tensor(np.asarray(a), dtype=dt, device=_dev())


def _solver(a):
    import torch

    import paper_1907_00072_gb300 as ppg

    return ppg.Solver(_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals, torch.float64))


def _time(fn, steps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(steps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def _relres(a, b, x):
    return float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b))


def run_c1(args):
    import torch

    import paper_1907_00072_gb300 as ppg

    a = w.c1_matrix()
    s = _solver(a)
    b = _T(w.rhs(a.n), torch.float64)
    v0 = _T(w.v0(a.n), torch.float64)
    res = {}
    for name, prec in (("f64", ppg.PPG_F64), ("f32", ppg.PPG_F32)):
        def step():
            s.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=v0)
            return s.solve(b, tol=1e-8, restart=50, maxit=5000, precision=prec)

        ms, (x, info) = _time(step, args.steps, args.warmup)
        res[name] = {"ms": round(ms, 3), "iterations": info.stats["iterations"],
                     "relres_host": _relres(a, w.rhs(a.n), x.cpu().numpy()),
                     "launches": info.stats["kernel_launches"]}
    print(json.dumps({"workload": "c1: 2D upwind 64^2 (n=4096), Pe 10, degree 10, GMRES(50), rtol 1e-8",
                      "unit": "ms", "results": res}))


def run_c3(args):
    import torch

    import paper_1907_00072_gb300 as ppg

    a = w.c3_matrix(args.N if args.N != 128 else 100)
    s = _solver(a)
    bh = w.rhs(a.n)
    b = _T(bh, torch.float64)
    v0 = _T(w.v0(a.n), torch.float64)
    res = {}
    xs = {}
    for name, prec in (("f32", ppg.PPG_F32), ("f64", ppg.PPG_F64)):
        def step():
            s.build_poly(25, ppg.PPG_BASIS_ROOTS, v0=v0)
            return s.solve(b, tol=1e-8, restart=50, maxit=5000, precision=prec)

        ms, (x, info) = _time(step, args.steps, args.warmup)
        xs[name] = x.cpu().numpy()
        res[name] = {"ms": round(ms, 3), "iterations": info.stats["iterations"], "restarts": info.stats["restarts"],
                     "relres_host": _relres(a, bh, xs[name]), "status": info.status}
    err = float(np.linalg.norm(xs["f32"] - xs["f64"]) / np.linalg.norm(xs["f64"]))
    print(json.dumps({"workload": f"c3: perturbed 27-point stencil, n={a.n}, nnz={a.nnz}, degree 25, GMRES(50)",
                      "unit": "ms", "results": res, "rel_error_f32_ir_vs_f64": err}))


def _peaks():
    try:
        return json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_c4(args):
    import torch

    import paper_1907_00072_gb300 as ppg

    t0 = time.perf_counter()
    specs = w.batch_specs()
    if getattr(args, "systems", 0):
        specs = specs[:args.systems]
    mats = [w.batch_system(i, side, pe) for i, (side, pe) in enumerate(specs)]
    gen_s = time.perf_counter() - t0
    systems = []
    for a, b in mats:
        systems.append((_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals, torch.float64),
                        _T(b, torch.float64), torch.zeros(a.n, dtype=torch.float64, device=_dev())))

    def step():
        for sy in systems:
            sy[4].zero_()
        return ppg.ppg_solve_batched(systems, degree=15, tol=1e-8, restart=30, maxit=20000, seed=2)

    ms, (status, stats) = _time(step, args.steps, max(args.warmup, 1))
    iters = [st["iterations"] for st in stats]
    rr = [_relres(a, b, sy[4].cpu().numpy()) for (a, b), sy in zip(mats, systems)]
    # the same systems solved one after another with the single-system solver (contexts made first)
    solvers = [ppg.Solver(sy[0], sy[1], sy[2]) for sy in systems]
    xs = [torch.zeros_like(sy[3]) for sy in systems]

    def seq():
        for i, (sv, sy) in enumerate(zip(solvers, systems)):
            sv.build_poly(15, ppg.PPG_BASIS_ROOTS, v0=None, seed=2 + i)
            xs[i].zero_()
            sv.solve(sy[3], x=xs[i], tol=1e-8, restart=30, maxit=20000, precision=ppg.PPG_F32)

    seq_ms = float("nan") if getattr(args, "systems", 0) else _time(seq, 1, 1)[0]
    total_n = sum(a.n for a, _ in mats)
    # algorithmic bytes of the batch (every matrix entry and vector once per pass): float64 construction
    # (d+1 SpMVs and the three basis passes per step), float32 iterations (d+1 SpMVs, passes over k+1,
    # k+2, k+2 and k+1 columns, the cycles' iterations taken as equal), float64 residuals, x updates
    d, m = 15, 30
    tot = 0.0
    for (a, _), st in zip(mats, stats):
        n, nnz = a.n, a.nnz
        sp64 = nnz * 12 + 4 * (n + 1) + 2 * n * 8
        sp32 = nnz * 8 + 4 * (n + 1) + 3 * n * 4
        tot += (d + 1) * sp64 + sum((4 * (j + 1) + 5) * n * 8 for j in range(d + 1))
        it, cyc = st["iterations"], max(st["restarts"], 1)
        tot += it * (d + 1) * sp32
        per = it / cyc
        tot += cyc * sum((4 * (j + 1) + 5) * n * 4 for j in range(int(round(per))))
        nres = st["spmvs"] - it * (d + 1) - (d + 1)
        tot += max(nres, 0) * (nnz * 12 + 4 * (n + 1) + 3 * n * 8) + cyc * (per * n * 4 + 2 * n * 8)
    pk = _peaks().get("hbm_gbs", 6800.0)
    gbs = tot / (ms * 1e-3) / 1e9
    # the tuner's choice of threads per row, by rows per CTA (the classes it tunes separately)
    cl = stats[0]["ctas_per_system"]
    lanes_by_class = {}
    for (a, _), st in zip(mats, stats):
        rpc = -(-a.n // cl)
        key = "<256" if rpc < 256 else ("<2048" if rpc < 2048 else ">=2048")
        lanes_by_class.setdefault(key, set()).add(int(st["spmv_lanes"]))
    lanes_by_class = {k: sorted(v) for k, v in lanes_by_class.items()}
    print(json.dumps({
        "workload": "c4: 256 x 2D upwind, sides log-uniform 32..448, Pe U[1,100], degree 15, GMRES(30), f32+f64 IR",
        "systems": len(systems), "total_rows": total_n, "total_nnz": sum(a.nnz for a, _ in mats),
        "batched_ms": round(ms, 3), "sequential_ms": None if seq_ms != seq_ms else round(seq_ms, 3),
        "speedup": None if seq_ms != seq_ms else round(seq_ms / ms, 2),
        "systems_per_s": round(len(systems) / (ms * 1e-3), 1), "status": status,
        "ctas_per_system": stats[0]["ctas_per_system"],
        "systems_by_ctas_per_system": {str(c): sum(1 for st in stats if st["ctas_per_system"] == c)
                                       for c in sorted({st["ctas_per_system"] for st in stats})},
        "spmv_lanes_by_rows_per_cta": lanes_by_class,
        "iterations_total": int(sum(iters)),
        "slowest_system_ms": round(max(st["spmv_ms"] for st in stats), 3),
        "last_start_ms": round(max(st["gs_ms"] for st in stats), 3),
        "iterations_min_max": [int(min(iters)), int(max(iters))], "relres_max_host": max(rr),
        "all_converged": bool(all(st["converged"] for st in stats)), "host_generation_s": round(gen_s, 2),
        "roofline": {"bound": "hbm", "kernel": "k_batch (one cluster per system)", "algorithmic_bytes": tot,
                     "achieved": round(gbs, 1), "peak": pk, "unit": "GB/s", "frac": round(gbs / pk, 3),
                     "note": "algorithmic bytes estimated from each system's iterations, cycles and SpMV count"}}))
    for sv in solvers:
        sv.close()


def run_c5(args):
    import torch

    import paper_1907_00072_gb300 as ppg

    a = w.c5_matrix()
    bh = w.rhs(a.n)
    xt = _T(w.uniform(w.SEED_XTARGET, a.n), torch.float64)
    s = _solver(a)
    s.build_poly(20, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n), torch.float64))
    roots = s.get_poly()[2]
    vals = s.vals.requires_grad_(True)  # the tensor the context was created from
    b = _T(bh, torch.float64).requires_grad_(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x = ppg.solve(s, vals, b, tol=1e-12, restart=50, maxit=3000)
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    e1.record()
    torch.cuda.synchronize()
    fwd_bwd_ms = e0.elapsed_time(e1)
    # a second forward/backward: the first includes building the transposed matrix
    e0.record()
    x = ppg.solve(s, vals, b, tol=1e-12, restart=50, maxit=3000)
    ((x - xt) ** 2).sum().backward()
    e1.record()
    torch.cuda.synchronize()
    fwd_bwd_ms2 = e0.elapsed_time(e1)
    vals.grad = None
    b.grad = None
    x = ppg.solve(s, vals, b, tol=1e-12, restart=50, maxit=3000)
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    _, finfo = s.solve(_T(bh, torch.float64), tol=1e-12, restart=50, maxit=3000)
    gb = b.grad.cpu().numpy()
    gv = vals.grad.cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e-6

    def L_b(bb):
        xx, _ = s.solve(_T(bb, torch.float64), tol=1e-12, restart=50, maxit=3000)
        return float(((xx - xt) ** 2).sum())

    errs_b = []
    for i in rng.choice(a.n, 50, replace=False):
        e = np.zeros(a.n)
        e[i] = h
        fd = (L_b(bh + e) - L_b(bh - e)) / (2 * h)
        errs_b.append(abs(fd - gb[i]) / max(abs(gb[i]), 1e-3 * np.abs(gb).max()))

    def L_vals(k, delta):
        v2 = a.vals.copy()
        v2[k] += delta
        a2 = w.CSR(a.n, a.rowptr, a.colidx, v2)
        s2 = _solver(a2)
        s2.set_poly(ppg.PPG_BASIS_ROOTS, roots)
        xx, _ = s2.solve(_T(bh, torch.float64), tol=1e-12, restart=50, maxit=3000)
        out = float(((xx - xt) ** 2).sum())
        s2.close()
        return out

    errs_v = []
    for k in rng.choice(a.nnz, 50, replace=False):
        fd = (L_vals(k, h) - L_vals(k, -h)) / (2 * h)
        errs_v.append(abs(fd - gv[k]) / max(abs(gv[k]), 1e-3 * np.abs(gv).max()))
    print(json.dumps({"workload": "c5: adjoint, 3D upwind 64^3 (n=262144), Pe 50, degree 20, L = ||x - x_t||^2",
                      "forward_backward_ms_first": round(fwd_bwd_ms, 3),
                      "forward_backward_ms": round(fwd_bwd_ms2, 3),
                      "forward_iterations": finfo.stats["iterations"], "forward_relres": finfo.stats["relres_true"],
                      "forward_status": finfo.status,
                      "fd_rel_err_db_max": max(errs_b), "fd_rel_err_db_median": statistics.median(errs_b),
                      "fd_rel_err_dvals_max": max(errs_v), "fd_rel_err_dvals_median": statistics.median(errs_v),
                      "samples": 50, "h": h,
                      "error_measure": "|fd - g_i| / max(|g_i|, 1e-3 max|g|)"}))


def run_ilu(args):
    """Section VI's composition on the 128^3 system: ILU(0) on the left alone (degree 0) against ILU(0)
    with a degree-12 polynomial on the right, float64 and float32 with float64 refinement; the
    polynomial without ILU(0) for context.  Time-to-solution per step = polynomial build + solve (the
    factorisation is set up once, its time reported apart)."""
    import torch

    import paper_1907_00072_gb300 as ppg

    a = w.c2_matrix(args.N)
    b = _T(w.rhs(a.n), torch.float64)
    v0 = _T(w.v0(a.n), torch.float64)
    s = _solver(a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_left_ilu0(1)
    setup_s = time.perf_counter() - t0
    res = {}
    for ilu in (1, 0):
        s.set_left_ilu0(ilu)
        for deg in ((0, 12) if ilu else (12,)):
            for pname, prec in (("f64", ppg.PPG_F64), ("f32", ppg.PPG_F32)):
                def step():
                    s.build_poly(deg, ppg.PPG_BASIS_ROOTS, v0=v0)
                    return s.solve(b, tol=1e-8, restart=50, maxit=5000, precision=prec)
                ms, (x, info) = _time(step, max(1, min(args.steps, 3)), 1)
                st = info.stats
                res[f"{'ilu_' if ilu else ''}d{deg}_{pname}"] = {
                    "ms": round(ms, 3), "iterations": st["iterations"], "restarts": st["restarts"],
                    "dots": st["dots"], "spmvs": st["spmvs"], "relres_true": st["relres_true"],
                    "status": info.status}
    print(json.dumps({"workload": "ILU(0) left + polynomial right (Section VI) on " + a.name + f" (n={a.n})",
                      "ilu_setup_s": round(setup_s, 3), "unit": "ms", "results": res}))
    s.close()


def run(args):
    {"c1": run_c1, "c3": run_c3, "c4": run_c4, "c5": run_c5, "ilu": run_ilu}[args.workload](args)
