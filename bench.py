#!/usr/bin/env python3
"""PP-GMRES time-to-solution on GB300 (one JSON line on stdout).

Workload: 3D convection-diffusion, 7-point upwind stencil on a 128^3 grid
(n = 2,097,152, nnz = 14,581,760, CSR float64), wind (1, 0.5, 0.25) scaled to
Peclet 50, b uniform in [-1, 1] (SplitMix64 seed 1), x0 = 0, GMRES(50), relative
residual 1e-8.  One step = build the minimum-residual polynomial (roots form,
v0 from seed 2) + solve, inputs resident in HBM.  The headline is the float32
p(A)/Arnoldi solve with float64 iterative refinement, its basis built in s-step
blocks of 4 Newton vectors (Section VII's combination of the polynomial with an
s-step method: the same GMRES iterates, three global reductions per block); the
solve without blocks (--sstep 0), the float64 solve and the other degrees are
reported under "variants".

  python bench.py [--gpus N --steps K --warmup W] [--degree D] [--precision f32|f64] [--sstep S]
  python bench.py --impl reference ...   # the CPU oracle: one full solve per step, same metric
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "PP-GMRES time-to-solution at rel. res. 1e-8; SpMV-chain HBM GB/s vs peak"
UNIT = "ms"
WORKLOAD = "3D convection-diffusion 7-point upwind, 128^3 (n=2097152, nnz=14581760), Pe 50, GMRES(50), rtol 1e-8"


def workload_name(N, nnz=None):
    if N == 128:
        return WORKLOAD
    return (f"3D convection-diffusion 7-point upwind, {N}^3 (n={N ** 3}" + (f", nnz={nnz}" if nnz else "")
            + "), Pe 50, GMRES(50), rtol 1e-8")


# DRAM traffic of a k_spmv_e<float> root step in place in the chain (C2 matrix; the mean of three
# consecutive root steps measured with ncu without flushing L2 between launches, so each link finds what
# the previous one left), summarised in profiles/k_spmv_c2_128cubed.md, and the kernel source it was taken
# with: when the source changes, the number no longer describes the kernel and the bench reports null.
SPMV_TRAFFIC = {"src_sha256_16": "3cf4760b97b8d7a7", "dram_bytes": round((56585728 + 41273088 + 28707328) / 3),
                "algorithmic_bytes": 112656384 + 16777216,
                "launch": "k_spmv_e root step in the running chain (tile-ELL values and window indices, x windows "
                          "staged in shared memory; write Y and P'); consecutive links walk their tiles in "
                          "opposite orders, so two thirds of the algorithmic bytes come from L2"}


def spmv_traffic():
    import hashlib

    src = os.path.join(ROOT, "paper_1907_00072_gb300", "csrc", "ppg_spmv.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None, None
    if sha != SPMV_TRAFFIC["src_sha256_16"]:
        return None, None
    return SPMV_TRAFFIC["dram_bytes"], SPMV_TRAFFIC


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples (every 100 ms, one streaming process) of SM clock and throttle reasons during
    the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._p = None
        self._t = None

    def _read(self):
        for line in self._p.stdout:
            parts = [s.strip() for s in line.strip().split(",")]
            if len(parts) >= 3:
                self.samples.append(parts)

    def __enter__(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                        "--format=csv,noheader,nounits", "-lms", "100"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._p = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        time.sleep(0.15)  # the first sample lands before the timed region starts
        return self

    def __exit__(self, *exc):
        if self._p is None:
            return
        self._p.terminate()
        try:
            self._p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self._p.kill()
        self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 3 + i and s[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ppg" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle


def oracle_solve(N, deg, with_x=False):
    """One full oracle time-to-solution on the benchmark workload (one host core): the polynomial
    of the given degree from the seeded v0, then MGS PP-GMRES(50) to relative residual 1e-8.
    Returns (seconds, iterations, relres, x or None)."""
    import oracle

    a = w.c2_matrix(N)
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    t0 = time.perf_counter()
    p = oracle.poly_gmres(a, v0, deg)
    r = oracle.gmres(a, b, p, tol=1e-8, m=50, maxit=20000)
    t1 = time.perf_counter()
    return t1 - t0, r.iters, r.relres, (r.x if with_x else None)


def run_reference(args, world, rank):
    """The reference arm: the oracle, as it stands, on the host cores.  Every step is one full
    time-to-solution (build + solve to 1e-8, one core each); the steps run as independent processes,
    at most --ref-workers at a time, so the run ends within a few minutes; each reports its own time."""
    if rank != 0:
        return
    import concurrent.futures as cf
    import multiprocessing as mp

    nsteps = args.warmup + args.steps
    workers = max(1, min(args.ref_workers, nsteps, os.cpu_count() or 1))
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(oracle_solve, [args.N] * nsteps, [args.degree] * nsteps))
    wall = time.perf_counter() - t0
    timed = res[args.warmup:]
    v = statistics.mean(t for t, _, _, _ in timed) * 1e3
    iters = timed[-1][1]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.N, w.expected_nnz_convdiff(args.N, 3)), "degree": args.degree,
                   "basis": "arnoldi-form (oracle)", "restart": 50},
        "iterations": iters, "relres_true": timed[-1][2],
        "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host_cores": os.cpu_count(), "concurrent_steps": workers,
                         "sample": f"full solve per step: oracle polynomial build (degree {args.degree}) + MGS "
                                   f"PP-GMRES(50) to relative residual 1e-8 ({iters} iterations), one core per "
                                   f"step, {workers} steps at a time on {os.cpu_count()} host cores"},
        "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "consistency": {"wall_s": round(wall, 1), "sum_of_step_seconds": round(sum(t for t, _, _, _ in res), 1)},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ppg", choices=["ppg", "reference"])
    ap.add_argument("--degree", type=int, default=10)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--N", type=int, default=128, help="grid side (128 is the benchmark workload)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-workers", type=int, default=8,
                    help="reference arm: full oracle solves run at once (one core each)")
    ap.add_argument("--profile-harness", action="store_true",
                    help="for ncu: build the polynomial and run --harness-iters iterations of one solve, print no "
                         "benchmark line")
    ap.add_argument("--harness-iters", type=int, default=20)
    ap.add_argument("--spmv-format", default="auto", choices=["auto", "csr", "sell", "staged"],
                    help="sparse format of the SpMV kernels (ppg_spmv_format)")
    ap.add_argument("--sstep", type=int, default=4,
                    help="s-step blocks of this many Newton vectors in the timed solve (Section VII's combination; "
                         "0: one basis vector per orthogonalisation)")
    ap.add_argument("--systems", type=int, default=0,
                    help="c4: solve only the first N systems of the batch (0: all 256), without the one-by-one "
                         "comparison when N > 0 (a small case for profiling)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "c4", "c5", "ilu"],
                    help="c2 (default): the benchmark line; c1/c3/c4/c5: the other configurations, one JSON line "
                         "each; ilu: ILU(0) on the left with and without the polynomial on the 128^3 system")
    args = ap.parse_args()

    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload != "c2":
        import other_workloads  # noqa: F401  (kept beside bench.py)

        other_workloads.run(args)
        return

    import torch

    import paper_1907_00072_gb300 as ppg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    a = w.c2_matrix(args.N)
    b_h = w.rhs(a.n)
    v0_h = w.v0(a.n)
    T = lambda x, dt=torch.float64: torch.as_tensor(x, dtype=dt, device=dev)  # noqa: E731
    s = ppg.Solver(T(a.rowptr, torch.int32), T(a.colidx, torch.int32), T(a.vals))
    s.spmv_format({"auto": ppg.PPG_SPMV_AUTO, "csr": ppg.PPG_SPMV_CSR, "sell": ppg.PPG_SPMV_SELL,
                   "staged": ppg.PPG_SPMV_STAGED}[args.spmv_format])
    b = T(b_h)
    v0 = T(v0_h)
    prec = ppg.PPG_F32 if args.precision == "f32" else ppg.PPG_F64
    stream = torch.cuda.current_stream()

    if args.profile_harness:
        s.build_poly(args.degree, ppg.PPG_BASIS_ROOTS, v0=v0)
        _, info = s.solve(b, tol=1e-8, restart=50, maxit=args.harness_iters, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile_harness": True, "iterations": info.stats["iterations"],
                          "launches": info.stats["kernel_launches"]}))
        s.close()
        return

    def step(deg=args.degree, precision=prec, bvec=b, f32_form=ppg.PPG_F32_FLEXIBLE, sstep=args.sstep):
        used, _ = s.build_poly(deg, ppg.PPG_BASIS_ROOTS, v0=v0)
        x, info = s.solve(bvec, tol=1e-8, restart=50, maxit=20000, precision=precision, f32_form=f32_form,
                          sstep=sstep, sstep_shift=1.0)
        return x, info

    for _ in range(args.warmup):
        x, info = step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            x, info = step()
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    # build_poly (roots form): v0 copy, norm, (d+1) x (SpMV + 3 Gram-Schmidt passes), roots
    build_launches = 2 + 4 * (args.degree + 1) + 1
    launches_per_step = int(np.mean([i.stats["kernel_launches"] for i in infos])) + build_launches
    last = infos[-1].stats

    # ---- end to end: pinned host b in, x out, through the public API
    b_pin = torch.from_numpy(b_h).pin_memory()
    x_pin = torch.empty(a.n, dtype=torch.float64).pin_memory()
    b_dev = torch.empty_like(b)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(args.steps):
        b_dev.copy_(b_pin, non_blocking=True)
        x, info = step(bvec=b_dev)
        x_pin.copy_(x, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e2.elapsed_time(e3) / args.steps, world, dev)
    relres_host = float(np.linalg.norm(b_h - a.to_scipy() @ x_pin.numpy()) / np.linalg.norm(b_h))

    # ---- roofline: one more (untimed) solve with the library's profiling on: CUDA events around
    # every SpMV-chain and Gram-Schmidt launch on the library's stream, with algorithmic bytes
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    # the timed configuration's solve (its SpMV chain is the dominant kernel; with s-step blocks its
    # "Gram-Schmidt" class holds the block passes, their reductions and finalisation, and the cycle ends)
    s.build_poly(args.degree, ppg.PPG_BASIS_ROOTS, v0=v0)
    _, pinfo = s.solve(b, tol=1e-8, restart=50, maxit=20000, precision=prec, profile=1, sstep=args.sstep or 4,
                       sstep_shift=1.0)
    ps = pinfo.stats
    spmv_gbs = ps["spmv_bytes"] / (ps["spmv_ms"] * 1e-3) / 1e9
    sps = ps
    sstep_gbs = sps["gs_bytes"] / (sps["gs_ms"] * 1e-3) / 1e9
    if not args.sstep:  # the timed configuration has no blocks: its own solve for the chain
        s.build_poly(args.degree, ppg.PPG_BASIS_ROOTS, v0=v0)
        _, pinfo = s.solve(b, tol=1e-8, restart=50, maxit=20000, precision=prec, profile=1)
        ps = pinfo.stats
        spmv_gbs = ps["spmv_bytes"] / (ps["spmv_ms"] * 1e-3) / 1e9
    # the two-pass classical Gram-Schmidt kernel of a solve without blocks
    s.build_poly(args.degree, ppg.PPG_BASIS_ROOTS, v0=v0)
    _, oinfo = s.solve(b, tol=1e-8, restart=50, maxit=20000, precision=prec, profile=1)
    ops = oinfo.stats
    gs_gbs = ops["gs_bytes"] / (ops["gs_ms"] * 1e-3) / 1e9
    # plain SpMV y = A x of the benchmark matrix, one event pair per launch
    dtype_t = torch.float32 if prec == ppg.PPG_F32 else torch.float64
    sv = 4 if prec == ppg.PPG_F32 else 8
    xs = torch.as_tensor(w.uniform(51, a.n), dtype=dtype_t, device=dev)
    ys = torch.empty_like(xs)
    for _ in range(3):
        s.spmv(xs, ys)
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for ea, eb in pairs:
        ea.record(stream)
        s.spmv(xs, ys)
        eb.record(stream)
    torch.cuda.synchronize()
    spmv_ms = statistics.mean(ea.elapsed_time(eb) for ea, eb in pairs)
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    idx_bytes = 2 if np.abs(a.colidx.astype(np.int64) - rows).max() <= 32767 else 4  # stored index format
    spmv_bytes = a.nnz * (sv + idx_bytes) + 4 * (a.n + 1) + 2 * a.n * sv

    x_bench = x.cpu().numpy()

    # ---- variants: degree x precision (x float32 form), one warm-up and five timed steps each
    variants = {}
    if not args.no_variants:
        forms = (("f64", ppg.PPG_F64, ppg.PPG_F32_FLEXIBLE), ("f32", ppg.PPG_F32, ppg.PPG_F32_FLEXIBLE),
                 ("f32_standard", ppg.PPG_F32, ppg.PPG_F32_STANDARD))
        # without blocks at every degree; s-step blocks (Section VII's combination, Newton shift 1) at the
        # headline degree
        runs = [(deg, pname, pv, form, 0) for deg in (1, 10, 25, 40) for pname, pv, form in forms]
        runs += [(args.degree, f"f32_sstep{k}", ppg.PPG_F32, ppg.PPG_F32_FLEXIBLE, k) for k in (2, 4, 5, 8)]
        runs += [(args.degree, "f32_standard_sstep4", ppg.PPG_F32, ppg.PPG_F32_STANDARD, 4)]
        runs += [(deg, "f32_sstep4", ppg.PPG_F32, ppg.PPG_F32_FLEXIBLE, 4) for deg in (25, 40)]
        runs += [(args.degree, "f64_sstep5", ppg.PPG_F64, ppg.PPG_F32_FLEXIBLE, 5)]
        for deg, pname, pv, form, sst in runs:
            step(deg, pv, f32_form=form, sstep=sst)
            ms_list = []
            for _ in range(5):
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                ea.record(stream)
                _, inf = step(deg, pv, f32_form=form, sstep=sst)
                eb.record(stream)
                torch.cuda.synchronize()
                ms_list.append(ea.elapsed_time(eb))
            variants[f"d{deg}_{pname}"] = {
                "ms_median": round(statistics.median(ms_list), 3), "ms_min": round(min(ms_list), 3),
                "ms_max": round(max(ms_list), 3), "repeats": len(ms_list),
                "iterations": inf.stats["iterations"], "restarts": inf.stats["restarts"],
                "relres_true": inf.stats["relres_true"], "dots": inf.stats["dots"], "status": inf.status}

    traffic, traffic_info = spmv_traffic()
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        # one full oracle solve (after the GPU work: no host load during the timed region)
        secs, it_o, rr_o, x_o = oracle_solve(args.N, args.degree, with_x=True)
        cpu = {"value": round(secs * 1e3, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
               "host_cores": os.cpu_count(),
               "sample": f"one full solve: oracle polynomial build (degree {args.degree}) + MGS PP-GMRES(50) to "
                         f"relative residual 1e-8 ({it_o} iterations) on one host core"}
        parity = {"oracle_iterations": it_o, "oracle_relres": rr_o, "iterations": last["iterations"],
                  "x_err_vs_oracle": float(np.linalg.norm(x_bench - x_o) / np.linalg.norm(x_o))}

    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == ppg.PPG_F32 else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.N, a.nnz), "degree": args.degree, "basis": "roots (Leja)",
                   "restart": 50,
                   "precision": ("f32 inner (flexible form, restart projection), f64 refinement" if prec == ppg.PPG_F32
                                 else "f64"),
                   "orthogonalisation": (f"s-step blocks of {args.sstep} Newton vectors (shift 1): block CGS2 + "
                                         f"Cholesky QR, 3 global reductions per block" if args.sstep
                                         else "two-pass classical Gram-Schmidt per basis vector"),
                   "sstep": args.sstep,
                   "l2": "working set of a step larger than L2 (matrix blocks 88 MB float32 + 117 MB "
                         "float64, basis up to 428 MB float32), no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": last["iterations"], "restarts": last["restarts"], "relres_true": last["relres_true"],
        "relres_host_check": relres_host,
        "roofline": {"bound": "hbm",
                     "kernel": ("k_spmv_e (tile-ELL blocks, x windows staged in shared memory)"
                                if prec == ppg.PPG_F32 and s.spmv_format() == ppg.PPG_SPMV_STAGED
                                else "k_spmv<float>" if prec == ppg.PPG_F32 else "k_spmv<double>")
                               + ": the SpMV chain, fused root steps of p(A) and the SpMV with A",
                     "achieved": round(spmv_gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(spmv_gbs / hbm, 3),
                     "peak_source": "measured" if "hbm_gbs" in pk else "fallback", "traffic": traffic,
                     "traffic_note": traffic_info,
                     "timed_segments": ps["spmv_segments"], "ms_total": round(ps["spmv_ms"], 3),
                     "bytes_total": ps["spmv_bytes"]},
        "roofline_ortho": {"bound": "hbm", "kernel": "k_gs (two-pass classical Gram-Schmidt, solve without blocks)",
                           "achieved": round(gs_gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gs_gbs / hbm, 3),
                           "timed_segments": ops["gs_segments"], "ms_total": round(ops["gs_ms"], 3),
                           "bytes_total": ops["gs_bytes"]},
        "roofline_sstep": {"bound": "hbm", "kernel": f"k_bgs_dot, k_bgs_finish, k_bgs_tri (s-step blocks of "
                                                     f"{args.sstep or 4} Newton vectors: block CGS2, Cholesky QR, "
                                                     f"Hessenberg recovery; cycle ends included)",
                           "achieved": round(sstep_gbs, 1), "peak": hbm, "unit": "GB/s",
                           "frac": round(sstep_gbs / hbm, 3), "timed_segments": sps["gs_segments"],
                           "ms_total": round(sps["gs_ms"], 3), "bytes_total": sps["gs_bytes"],
                           "solve_ms": round(sps["time_ms"], 3), "iterations": sps["iterations"],
                           "global_reductions": sps["dots"]},
        "spmv_plain": {"achieved": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                       "ms_per_launch": round(spmv_ms, 5), "bytes_per_launch": spmv_bytes},
        "cpu_baseline": cpu,
        "parity": parity,
        "e2e": {"value": round(e2e_ms, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * a.n, "d2h_bytes_per_step": 8 * a.n},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "variants": variants,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
