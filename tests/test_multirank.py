"""The multi-GPU form of the benchmark, on the CPU: one process per rank
(torch.distributed, gloo, world size 2).  The path shards into independent
replicas (every rank evaluates the same sweep on its own GPU; no data
exchange), so the only cross-rank steps are the barrier and the maximum of
the ranks' times; the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    worst = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (worst, bench.job_gevals(880e6, 5, world, worst))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # both ranks' evaluations over the slowest rank's time
    assert res[0][1] == pytest.approx(2 * 880e6 * 5 / 0.150 / 1e9)
    assert bench.max_over_ranks(123.0) == 123.0


def test_reference_arm_two_ranks():
    """Under torchrun with two ranks the reference arm prints one line, from
    rank 0, and both ranks exit 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--ref-per-v", "20"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    # rank 0 alone ran the oracle: the value is not a whole-job figure
    assert d["ranks_used"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle"
