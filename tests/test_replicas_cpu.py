"""The multi-GPU form's host logic on CPU: two `gloo` ranks (world size 2).

Replicas share nothing on the data path; the only collectives are the barrier and the maximum
of the per-rank step times, from which the whole-job throughput is formed.  Also checks that
the reference arm under a 2-rank launch prints one line, from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

from paper_1104_0672_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    w, r, local = replicas.env()
    dist = replicas.init(w, "gloo")
    try:
        dist.barrier()
        # rank r "took" 10 + 5 r ms per step
        ms = replicas.max_over_ranks(10.0 + 5.0 * r, dist)
        results[r] = (w, r, local, replicas.map_config(r), ms,
                      replicas.job_throughput(1_000_000, w, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(results)
    assert sorted(res) == [0, 1]
    for r, (w, rr, local, cfg, ms, gpx) in res.items():
        assert (w, rr, local) == (2, r, r)
        assert ms == 15.0                       # the slowest rank bounds the job
        assert gpx == pytest.approx(2 * 1_000_000 / 15e-3 / 1e9)
    assert res[0][3] != res[1][3]               # replicas convolve different maps


def test_single_process_needs_no_group():
    assert replicas.init(1, "gloo") is None
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(50_331_648 * 16, 1, 20.0) == pytest.approx(40.265, rel=1e-4)


def test_reference_arm_under_two_ranks_prints_once():
    """bench.py --impl reference launched as 2 ranks: rank 0 times the oracle and prints one
    JSON line, rank 1 exits 0 without work (small grid, so the oracle sample takes seconds)."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--nside", "32", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
