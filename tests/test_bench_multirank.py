"""Host logic of the multi-process bench path (world_size 2, gloo on CPU).

On N GPUs the benchmark runs one replica per GPU (the Hessian-product blocks of
independent problems shard with no exchange), times each rank with device
events, and reports the slowest rank's time and the units of all ranks. These
tests cover the pieces that need no GPU: the max-over-ranks reduction, the
whole-job throughput and the launch contract of the CPU reference arm under
torchrun (rank 0 alone prints one JSON line)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(dist, times[rank], torch.device("cpu"))
        v = bench.job_throughput(128 * 5, world, t / 1e3)
        out_q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world, port = 2, _free_port()
    times = [812.5, 1030.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == max(times)                       # every rank sees the slowest rank's time
        assert v == pytest.approx(128 * 5 * world / (max(times) / 1e3))


def test_single_process_helpers():
    assert bench.max_over_ranks(None, 3.5, None) == 3.5
    assert bench.job_throughput(10, 1, 2.0) == 5.0


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"


def test_paper_counts_tables():
    """The paper's printed PDE-solve counts the experiment arms compare against
    (Tables 3 and 4): every method, in the column order of the comparison rows."""
    t3, t4 = bench.paper_counts("T3"), bench.paper_counts("T4")
    assert set(t3) == {"Prec_Gamma", "Prec_Lanczos", "SketchPrec_RandSVD", "SketchPrec_Nystrom",
                       "SketchPrec_SingleView", "SketchSolv_RandSVD", "SketchSolv_Nystrom",
                       "SketchSolv_SingleView"}
    assert set(t4) == {"Prec_Gamma", "SketchPrec_RandSVD", "SketchPrec_Nystrom", "SketchPrec_SingleView",
                       "SketchPrecA_RandSVD", "SketchPrecA_Nystrom", "SketchPrecA_SingleView"}
    assert t3["SketchSolv_SingleView"] == [None, 45, 93, 10, 0, 3]
    assert t4["Prec_Gamma"] == [15441, None, None, 57, 15441, 15466]
    # Table 4 accounting: online ADJ = PCG iterations + 25 GN gradients (+ 1 where printed so)
    for name, row in t4.items():
        assert row[5] - row[0] in (25, 26), name
