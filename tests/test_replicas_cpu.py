"""The multi-GPU form's host logic on CPU: two `gloo` ranks (world size 2).

Replicas share nothing on the forward data path; the collectives are the barrier, the maximum
of the per-rank step times, from which the whole-job throughput is formed, and the sum of a
shared beam's knot gradient over the ranks after the backward pass.  Also checks that the
reference arm under a 2-rank launch prints one line, from rank 0."""
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


def _knot_rank_main(rank, world, port, results):
    """Rank r holds map r of a shared-beam fit; its knot gradient comes from the FP64 oracle
    (the gradient the GPU backward pass reproduces) and is summed over the ranks."""
    import numpy as np
    import torch

    import oracle
    from paper_1104_0672_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    w, r, _ = replicas.env()
    dist = replicas.init(w, "gloo")
    try:
        grid, nside = ("healpix", 4), 4
        gmax = 40 * inputs.DEG
        knots = inputs.gaussian_knots(15 * inputs.DEG, gmax, 24)
        x = inputs.white_noise(12 * nside * nside, 1, config=21, salt=r)[0].astype(np.float64)
        g = inputs.white_noise(12 * nside * nside, 1, config=22, salt=r)[0].astype(np.float64)
        local = oracle.knot_grad(grid, knots, gmax, x, g)
        gk = torch.from_numpy(local.copy())[None]
        replicas.allreduce_knot_grad(gk, dist)
        results[r] = (local, gk[0].numpy())
    finally:
        dist.destroy_process_group()


def test_shared_beam_knot_gradient_summed_over_ranks():
    """The all-reduced knot gradient on every rank equals the derivative of the summed loss
    J(f) = sum_r <g_r, L(f) x_r> over both ranks' maps, taken by central differences of the
    oracle's forward convolution (exact up to rounding: L is linear in the knots)."""
    import numpy as np

    import oracle
    from paper_1104_0672_gb300 import inputs
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_knot_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(results)
    total0, total1 = res[0][1], res[1][1]
    assert np.array_equal(total0, total1)                       # every rank holds the sum
    assert not np.allclose(res[0][0], res[1][0])                # the ranks' own parts differ
    np.testing.assert_allclose(total0, res[0][0] + res[1][0], rtol=0, atol=1e-15 * np.abs(total0).max())
    grid, nside = ("healpix", 4), 4
    gmax = 40 * inputs.DEG
    knots = inputs.gaussian_knots(15 * inputs.DEG, gmax, 24)
    maps = [(inputs.white_noise(12 * nside * nside, 1, config=21, salt=r)[0].astype(np.float64),
             inputs.white_noise(12 * nside * nside, 1, config=22, salt=r)[0].astype(np.float64))
            for r in range(2)]

    def loss(f):
        return sum(float(np.dot(g, oracle.convolve(grid, f, gmax, x))) for x, g in maps)

    for t in (0, 5, 11, 17):
        e = np.zeros_like(knots)
        e[t] = 1.0
        fd = (loss(knots + e) - loss(knots - e)) / 2.0
        assert abs(fd - total0[t]) <= 1e-10 * max(1.0, np.abs(total0).max())


def test_single_process_needs_no_group():
    assert replicas.init(1, "gloo") is None
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(50_331_648 * 16, 1, 20.0) == pytest.approx(40.265, rel=1e-4)
    import torch
    gk = torch.arange(4, dtype=torch.float64)
    assert replicas.allreduce_knot_grad(gk) is gk and gk.tolist() == [0.0, 1.0, 2.0, 3.0]


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
