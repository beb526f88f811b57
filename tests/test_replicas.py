"""The N > 1 path: independent replicas coordinated on the host only
(barrier, max and sum over ranks), run as two gloo ranks on the CPU, and the
reference arm of bench.py under torchrun with two ranks (rank 0 alone
prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2104_05615_gb300.replicas import Replicas
    rep = Replicas("gloo")
    rep.barrier()
    res = {"max": rep.max(0.5 + rank), "sum": rep.sum(1.0 + rank), "rank": rep.rank, "world": rep.world}
    rep.barrier()
    rep.close()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_replicas_gloo_two_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["rank"] == r and d["world"] == 2
        assert d["max"] == 1.5          # slowest rank's time
        assert d["sum"] == 3.0          # units of the whole job


def test_replicas_single_process_is_identity():
    from paper_2104_05615_gb300.replicas import Replicas
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK") if k in os.environ}
    try:
        rep = Replicas("gloo")
        assert rep.world == 1 and rep.max(2.5) == 2.5 and rep.sum(4.0) == 4.0
        rep.barrier()
        rep.close()
    finally:
        os.environ.update(env)


def test_reference_arm_two_ranks_rank0_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--config", "C1", "--steps", "1", "--warmup", "1", "--ref-iters", "10"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
