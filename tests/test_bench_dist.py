"""Multi-process paths of bench.py on CPU (gloo, world size 2): the rank helpers
(barrier, max over ranks) and the reference arm, which only rank 0 runs."""
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


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(impl="reference")
    r, w, _ = bench.dist_setup(args)
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + r, w)
    bench.barrier(w)
    import torch.distributed as dist

    dist.destroy_process_group()
    q.put((r, w, m))


def test_rank_helpers_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2, 2.5), (1, 2, 2.5)]


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_line_under_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--workload", "small"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_search_traffic_only_for_the_captured_source(monkeypatch):
    """The roofline's DRAM traffic is reported per pass for the scene it was
    captured on, and only while the solver source has the captured hash."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.search_traffic_per_launch("lobes", 7) is None
    got = bench.search_traffic_per_launch("earthquake", 7)
    import hashlib

    with open(os.path.join(ROOT, "paper_2609_36267_b300", "csrc", "ww_mcf.cu"), "rb") as f:
        same = hashlib.sha256(f.read()).hexdigest() == bench.SEARCH_DRAM_SOURCE_SHA256
    assert got == (bench.SEARCH_DRAM_BYTES_PER_UNWRAP / 7 if same else None)
    monkeypatch.setattr(bench, "SEARCH_DRAM_SOURCE_SHA256", "0" * 64)
    assert bench.search_traffic_per_launch("earthquake", 7) is None
