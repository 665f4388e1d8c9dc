"""The N > 1 path on CPU: gloo process groups of world size 2 (replicas only;
no data-path collective exists, only the measurement's barrier and max)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_1512_01977_gb300 import replicas

    rep = replicas.Replicas(backend="gloo")
    rep.barrier()
    slow = rep.max(1.0 + rank)  # rank r "took" 1 + r seconds
    rate = replicas.aggregate_rate(1000.0, ws, slow)
    out.put((rank, slow, rate))
    rep.close()


def test_max_and_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate in res:
        assert slow == 2.0  # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_process_replicas_are_a_no_op(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    from paper_1512_01977_gb300 import replicas

    rep = replicas.Replicas(backend="gloo")
    assert not rep.active
    rep.barrier()
    assert rep.max(3.5) == 3.5
    rep.close()


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched as two ranks: rank 0 alone runs the
    oracle and prints the JSON line, the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "MLUPS" and d["value"] > 0
