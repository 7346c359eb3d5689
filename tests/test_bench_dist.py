"""Multi-process paths of bench.py on CPU (gloo, world size 2).

The GPU arm runs one independent replica per rank (bodies do not interact),
so the only cross-rank operations are a barrier and the reductions that turn
per-rank times into the whole-job rate: units summed over ranks, time the
slowest rank's.  The reference arm runs on rank 0 alone.
"""
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


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_path):
    # CPU ranks even on a machine with a GPU (bench picks gloo without CUDA)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    wsz, r, _ = bench.dist_setup()
    assert (wsz, r) == (ws, rank)
    bench.barrier(wsz)
    # rank r processed 1000 * (r + 1) units in (r + 1) * 10 ms per step
    value, t_max = bench.job_rate(wsz, 1000 * (rank + 1), 4, 10.0 * (rank + 1), "cpu")
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"value": value, "t_max": t_max}, f)
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks(tmp_path):
    out = tmp_path / "rate.json"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True,
                       start_method="spawn")
    got = json.loads(out.read_text())
    assert got["t_max"] == pytest.approx(20.0)
    # (1000 + 2000) units x 4 steps / 20 ms
    assert got["value"] == pytest.approx(3000 * 4 / 20e-3)


def test_reference_arm_prints_one_line_from_rank_zero():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "drop64"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
