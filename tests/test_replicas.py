"""The N>1 path of bench.py on CPU: independent replicas, gloo, world size 2.

The method is run as one independent solve per GPU (replicas: no data-path
collective), so what needs checking on more than one process is the host
logic around it: process-group setup from the torchrun environment, the
barrier, the max-over-ranks timing, and that only rank 0 prints a line.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import types

    import bench

    args = types.SimpleNamespace(impl="reference")
    w, r, local = bench.dist_init(args)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # each rank "measured" a different time; every rank must see the largest
    m = bench.max_over_ranks(10.0 + 3.5 * rank, w)
    bench.barrier(w)
    import torch.distributed as dist

    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "max": m}, f)


def test_dist_helpers_world2(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["rank"] for x in res] == [0, 1]
    assert all(x["world"] == 2 and x["max"] == 13.5 for x in res)


def test_single_process_helpers_are_noops():
    sys.path.insert(0, ROOT)
    import types

    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        assert k not in os.environ or os.environ[k] in ("0", "1")
    w, r, local = bench.dist_init(types.SimpleNamespace(impl="reference"))
    assert (w, r, local) == (1, 0, 0)
    bench.barrier(1)
    assert bench.max_over_ranks(2.5, 1) == 2.5


def test_reference_arm_under_torchrun_world2():
    """`bench.py --impl reference` launched as the driver launches it for N=2: rank 0 alone prints one line."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--N", "10", "--degree", "4", "--ref-workers", "2"]
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "10^3" in d["config"]["workload"]
    assert "full solve" in d["cpu_baseline"]["sample"] and d["iterations"] > 0 and d["relres_true"] <= 1e-8
