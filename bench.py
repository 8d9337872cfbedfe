#!/usr/bin/env python3
"""Benchmark of the GB300 ring-band sphere convolution (hybrid method of Elsner & Wandelt 2011).

Default workload (one step = one full forward pass of the hot path over one batch):
HEALPix nside 2048 (50,331,648 px), 16 FP32 white-noise maps, one shared Gaussian beam of
5' FWHM tabulated at 256 knots with 15' support; ring FFTs, FP64 kernel sampling, fused
coefficient generation + ring-band contraction, fold + inverse FFTs, pole-ring fix.

Prints one JSON line.  `value` is Gpix*maps/s with maps resident in HBM; `e2e` is the same
metric through the public API with pinned host buffers (host->device copy of the maps and
device->host copy of the result inside the timed region).  `roofline` is the dominant
kernel against its bound; `step_roofline` the whole step, T_roof = max(map bytes / HBM, sum of
the FFT, contraction and generation flops over their unit peaks), as frac = T_roof / T_step.
The 3.2 GB of maps per step are larger than the 129 MB L2, so no explicit flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--nside 2048] [--nmaps 16] [--beams shared|permap]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpix·maps/s at nside 2048 FWHM 5′, batched TF32 vs plain FP32, ≤1e-5 frac RMS"
UNIT = "Gpix·maps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--nside", type=int, default=2048)
    p.add_argument("--nmaps", type=int, default=16)
    p.add_argument("--beams", default="shared", choices=["shared", "permap"])
    p.add_argument("--form", default="tf32", choices=["tf32", "fp32"],
                   help="tf32: tensor-core 3xTF32 coefficient generation; fp32: CUDA cores")
    p.add_argument("--no-compare", action="store_true", help="skip timing the other form")
    p.add_argument("--fwhm-arcmin", type=float, default=5.0)
    p.add_argument("--support-arcmin", type=float, default=15.0)
    p.add_argument("--knots", type=int, default=256)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    p.add_argument("--e2e-chunk", type=int, default=2, help="maps per chunk of the host-buffer pipeline")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def workload_name(a):
    beams = "one shared beam" if a.beams == "shared" else "per-map beams FWHM U[4.5',5.5']"
    form = "batched 3xTF32 tensor-core form" if a.form == "tf32" else "plain FP32 form"
    return (f"HEALPix nside {a.nside}, {a.nmaps} FP32 white-noise maps, Gaussian FWHM "
            f"{a.fwhm_arcmin:g}' support {a.support_arcmin:g}' {a.knots} knots, {beams}, "
            f"{form}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        inside = [r for (t, r) in self.rows if any(a - 0.25 <= t <= b + 0.25 for a, b in self.windows)]
        use = inside or [r for _, r in self.rows]
        sm = [float(r[1]) for r in use if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(use), "samples_in_timed_window": len(inside)}


# ------------------------------------------------------------------ oracle baseline
def oracle_sample(nside, knots, gmax, rings_per_step=4):
    """The FP64 oracle on a bounded sample of the workload: `rings_per_step` consecutive
    equatorial output rings of map 0 (it transforms every input ring they need)."""
    import oracle
    from paper_1104_0672_gb300 import inputs
    oracle.build()
    x = inputs.white_noise(12 * nside * nside, 1, config=3)[0].astype(np.float64)
    c = 2 * nside - 1
    rings = list(range(c - rings_per_step // 2, c - rings_per_step // 2 + rings_per_step))
    th, ph, w, n, off = oracle.geometry(("healpix", nside))
    px = int(sum(n[i] for i in rings))
    cores = os.cpu_count() or 1

    def run():
        t0 = time.perf_counter()
        oracle.convolve(("healpix", nside), knots, gmax, x, rings=rings, nthreads=cores)
        return time.perf_counter() - t0
    desc = (f"{rings_per_step} consecutive equatorial output rings ({px} px) of one map, "
            f"FP64 naive-DFT oracle incl. the DFTs of every input ring they need")
    return run, px, cores, desc


# DRAM bytes (read + write) per launch of a stage's kernel, from one ncu capture (a 4-map case
# scaled to 16 maps by the map count), valid only for the CUDA sources the kernel is built from
# (its translation unit and the headers it includes): any change to them reports null until
# the capture is redone.
TRAFFIC = {
    "fft_inv": {"bytes_per_launch": 1.99966e9, "nmaps": 16, "nside": 2048,
                "sources": ["ring_fft_inv.cu", "ring_common.cuh", "fft_engine.cuh", "device_common.cuh",
                            "arkcos_impl.cuh", "arkcos.h"],
                "sources_sha256": "f7c5f081d237ef821a669d0c725d69d36ee9116053f3f694bc0785ee6e2f842f"},
}


def measured_units(ark):
    """Arithmetic peaks of this GPU from the library's isolated kernels (best of five launches
    each): FP32 FMA (the larger of scalar and packed two-lane), FP64 FMA, tcgen05 kind::tf32."""
    fp32 = max(ark.measure_peak("fp32")["tflops"], ark.measure_peak("fp32x2")["tflops"])
    return {"fp32_tflops": fp32, "fp64_tflops": ark.measure_peak("fp64")["tflops"],
            "tf32_mma_tflops": ark.measure_peak("tf32_mma")["tflops"]}


def sources_digest(names) -> str:
    import hashlib
    h = hashlib.sha256()
    here = os.path.dirname(os.path.abspath(__file__))
    for n in names:
        p = os.path.join(here, "include", n) if n.endswith(".h") else \
            os.path.join(here, "paper_1104_0672_gb300", "csrc", n)
        h.update(n.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1104_0672_gb300 import inputs
    gmax = a.support_arcmin * inputs.ARCMIN
    knots = inputs.gaussian_knots(a.fwhm_arcmin * inputs.ARCMIN, gmax, a.knots)
    run, px, cores, desc = oracle_sample(a.nside, knots, gmax)
    for _ in range(a.warmup):
        run()
    ts = [run() for _ in range(a.steps)]
    t = sum(ts) / len(ts)
    v = px / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a) + " (oracle on a bounded sample per step)",
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GB300 arm
def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    import paper_1104_0672_gb300 as ark
    from paper_1104_0672_gb300 import inputs

    from paper_1104_0672_gb300 import replicas

    world, rank, local = replicas.env()
    if world > 1:
        torch.cuda.set_device(local)
    dist = replicas.init(world, "nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    grid = ark.Grid.healpix(a.nside)
    gmax = a.support_arcmin * inputs.ARCMIN
    if a.beams == "shared":
        kernels = [ark.Kernel(grid, inputs.gaussian_knots(a.fwhm_arcmin * inputs.ARCMIN, gmax,
                                                          a.knots), gmax)]
    else:
        fw = inputs.rng(4, 1).uniform(4.5, 5.5, a.nmaps)
        kernels = [ark.Kernel(grid, inputs.gaussian_knots(f * inputs.ARCMIN, 3 * f * inputs.ARCMIN,
                                                          a.knots), 3 * f * inputs.ARCMIN)
                   for f in fw]
    kk = kernels[0] if len(kernels) == 1 else kernels
    B = a.nmaps
    x_host = torch.from_numpy(inputs.white_noise(grid.npix, B, config=replicas.map_config(rank))).pin_memory()
    x = x_host.to(dev)
    y = torch.empty_like(x)
    ws = torch.empty(ark.workspace_size(grid, kk, B), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    flags = ark.FLAG_3XTF32 if a.form == "tf32" else 0

    def step(fl=None):
        ark.convolve(grid, kk, x, out=y, workspace=ws, flags=flags if fl is None else fl)

    # launch shapes chosen once by the library's autotuner on these buffers (untimed), and the
    # arithmetic peaks of this GPU (roofline denominators, untimed)
    tuned = None if a.no_autotune else ark.autotune(grid, kk, x, flags=flags, out=y, workspace=ws)
    units = measured_units(ark)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ark.stage_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    clocks.mark(t_wall0, t_wall1)
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    stages = ark.stage_report()
    ark.stage_timing(False)
    ms = replicas.max_over_ranks(ms_total / a.steps, dist, dev)
    pix = B * grid.npix * world
    value = replicas.job_throughput(B * grid.npix, world, ms)

    # end-to-end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        # the host-buffer entry point: uploads, convolutions and downloads of chunks of maps
        # overlap on three streams
        out_host = torch.empty_like(x_host).pin_memory()
        wsh = torch.empty(ark.host_workspace_size(grid, kk, B, a.e2e_chunk, flags), dtype=torch.uint8, device=dev)
        for _ in range(2):
            ark.convolve_host(grid, kk, x_host, out=out_host, maps_per_chunk=a.e2e_chunk, workspace=wsh,
                              flags=flags)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        n_e2e = max(3, min(a.steps, 10))
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        f0.record(stream)
        for _ in range(n_e2e):
            ark.convolve_host(grid, kk, x_host, out=out_host, maps_per_chunk=a.e2e_chunk, workspace=wsh,
                              flags=flags)
        f1.record(stream)
        torch.cuda.synchronize()
        clocks.mark(tw0, time.time())
        ms_e2e = replicas.max_over_ranks(f0.elapsed_time(f1) / n_e2e, dist, dev)
        nb = B * grid.npix * 4
        e2e = {"value": pix / (ms_e2e * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb, "ms_per_step": ms_e2e, "maps_per_chunk": a.e2e_chunk,
               "api": "arkcos_convolve_host (pinned host buffers)"}
        del wsh
    # the other form of the coefficient generation, same workload, for comparison
    other = None
    if not a.no_compare:
        ofl = 0 if a.form == "tf32" else ark.FLAG_3XTF32
        for _ in range(2):
            step(ofl)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        g0.record(stream)
        for _ in range(a.steps):
            step(ofl)
        g1.record(stream)
        torch.cuda.synchronize()
        clocks.mark(tw0, time.time())
        ms_o = g0.elapsed_time(g1) / a.steps
        other = {"form": "fp32" if a.form == "tf32" else "tf32",
                 "value": B * grid.npix * world / (ms_o * 1e-3) / 1e9, "ms_per_step": ms_o}
    # extra measurements on the same maps: one beam per map (FWHM U[4.5', 5.5'], support 3 FWHM),
    # both forms, and the backward pass (map and knot gradients) with the shared beam
    extras = {}
    if not a.no_compare and a.beams == "shared":
        fw = inputs.rng(4, 1).uniform(4.5, 5.5, B)
        pk_list = [ark.Kernel(grid, inputs.gaussian_knots(f * inputs.ARCMIN, 3 * f * inputs.ARCMIN, a.knots),
                              3 * f * inputs.ARCMIN) for f in fw]
        wsp = torch.empty(ark.workspace_size(grid, pk_list, B), dtype=torch.uint8, device=dev)
        for name, fl in (("tf32", ark.FLAG_3XTF32), ("fp32", 0)):
            ark.convolve(grid, pk_list, x, out=y, workspace=wsp, flags=fl)
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tw0 = time.time()
            h0.record(stream)
            nrep = 3
            for _ in range(nrep):
                ark.convolve(grid, pk_list, x, out=y, workspace=wsp, flags=fl)
            h1.record(stream)
            torch.cuda.synchronize()
            clocks.mark(tw0, time.time())
            msp = h0.elapsed_time(h1) / nrep
            extras["per_map_beams_" + name] = {"value": B * grid.npix * world / (msp * 1e-3) / 1e9,
                                               "ms_per_step": msp}
        del wsp, pk_list
        # the BASIC variant (ring-Nyquist truncation instead of the periodic extension, Sec. 4.1)
        # on the same maps and beam: the cost ratio of the ENHANCED form
        ark.convolve(grid, kk, x, out=y, workspace=ws, flags=flags | ark.FLAG_BASIC)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        h0.record(stream)
        for _ in range(3):
            ark.convolve(grid, kk, x, out=y, workspace=ws, flags=flags | ark.FLAG_BASIC)
        h1.record(stream)
        torch.cuda.synchronize()
        clocks.mark(tw0, time.time())
        msb = h0.elapsed_time(h1) / 3
        extras["basic_variant"] = {"value": B * grid.npix * world / (msb * 1e-3) / 1e9, "ms_per_step": msb,
                                   "enhanced_over_basic_time": ms / msb}
        wsb = torch.empty(ark.workspace_size(grid, kk, B, flags, True), dtype=torch.uint8, device=dev)
        ark.convolve_backward(grid, kk, x, y, flags=flags, workspace=wsb)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        h0.record(stream)
        for _ in range(2):
            ark.convolve_backward(grid, kk, x, y, flags=flags, workspace=wsb)
        h1.record(stream)
        torch.cuda.synchronize()
        clocks.mark(tw0, time.time())
        msb = h0.elapsed_time(h1) / 2
        extras["backward_map_and_knot_gradients"] = {"value": B * grid.npix * world / (msb * 1e-3) / 1e9,
                                                     "ms_per_step": msb}
        del wsb
        # ten Gaussian components (4.5'-5.22', support 3 FWHM) of one asymmetric-beam
        # decomposition on one map (Sec. 5): one multi-kernel call with the weighted sum against
        # ten single calls
        fw10 = 4.5 + 0.08 * np.arange(10)
        k10 = [ark.Kernel(grid, inputs.gaussian_knots(f * inputs.ARCMIN, 3 * f * inputs.ARCMIN, a.knots),
                          3 * f * inputs.ARCMIN) for f in fw10]
        w10 = inputs.rng(33).uniform(0.2, 1.0, 10)
        x1 = x[:1]
        y1 = torch.empty_like(x1)
        wsm = torch.empty(ark.multi_workspace_size(grid, k10, 1, True, flags), dtype=torch.uint8, device=dev)
        ws1 = torch.empty(max(ark.workspace_size(grid, kq, 1, flags) for kq in k10), dtype=torch.uint8, device=dev)

        def multi():
            ark.convolve_multi(grid, k10, x1, weights=w10, flags=flags, out=y1, workspace=wsm)

        def singles():
            for kq in k10:
                ark.convolve(grid, kq, x1, flags, out=y1, workspace=ws1)
        for name, fn in (("multi_kernel_10_weighted", multi), ("single_calls_10", singles)):
            fn()
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tw0 = time.time()
            h0.record(stream)
            for _ in range(3):
                fn()
            h1.record(stream)
            torch.cuda.synchronize()
            clocks.mark(tw0, time.time())
            extras[name] = {"ms_per_call": h0.elapsed_time(h1) / 3, "maps": 1, "kernels": 10}
        extras["multi_kernel_10_weighted"]["speedup_vs_single_calls"] = (
            extras["single_calls_10"]["ms_per_call"] / extras["multi_kernel_10_weighted"]["ms_per_call"])
        del wsm, ws1, k10
    # config 4: 64 HEALPix nside 1024 maps, one Gaussian beam per map (FWHM U[4.5', 10'], support
    # 3 FWHM), autotuned, captured once into a CUDA graph and replayed
    if not a.no_compare and a.beams == "shared":
        g4 = ark.Grid.healpix(1024)
        f4 = inputs.rng(4, 0).uniform(4.5, 10.0, 64)
        k4 = [ark.Kernel(g4, inputs.gaussian_knots(f * inputs.ARCMIN, 3 * f * inputs.ARCMIN, a.knots),
                         3 * f * inputs.ARCMIN) for f in f4]
        x4 = torch.from_numpy(inputs.white_noise(g4.npix, 64, config=4)).to(dev)
        y4 = torch.empty_like(x4)
        ws4 = torch.empty(ark.workspace_size(g4, k4, 64, flags), dtype=torch.uint8, device=dev)
        shape4 = ark.autotune(g4, k4, x4, flags=flags, out=y4, workspace=ws4)
        ark.convolve(g4, k4, x4, flags, out=y4, workspace=ws4)
        torch.cuda.synchronize()
        graph4 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph4):
            ark.convolve(g4, k4, x4, flags, out=y4, workspace=ws4)
        graph4.replay()
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        h0.record(stream)
        for _ in range(5):
            graph4.replay()
        h1.record(stream)
        torch.cuda.synchronize()
        clocks.mark(tw0, time.time())
        ms4 = h0.elapsed_time(h1) / 5
        extras["config4_64maps_nside1024_per_map_beams_graph"] = {
            "value": 64 * g4.npix * world / (ms4 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms4,
            "launch_shape": shape4, "form": "3xtf32-tensor-core" if a.form == "tf32" else "plain-fp32"}
        del graph4, x4, y4, ws4, k4
    ark.sync_status()
    clocks.stop()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (per-launch algorithmic work / CUDA-event duration), against
    # the measured HBM copy bandwidth (MEASURED_PEAKS.json) or the arithmetic peaks measured above
    pk, pk_src = peaks()
    NH = grid.nlon // 2 + 1
    pairs = sum(ark.kernel_info(k)[0] for k in kernels)
    samples = sum(ark.kernel_info(k)[1] for k in kernels)
    nspec = (grid.npix + 2 * grid.nrings) // 2  # compact half spectra: sum over rings of n/2 + 1
    fp32 = units["fp32_tflops"]
    tf32x3 = units["tf32_mma_tflops"] / 3.0  # three TF32 products per FP32 product
    stage_rows = {}
    for name, (sms, ex, nl) in stages.items():
        per_launch_ms = sms / max(nl, 1)
        if name == "contract":
            # generation: 2 flop per (sample, mode) per beam, on the tensor cores in the 3xTF32
            # form; contraction: 8 flop per (ring pair, mode, map) (complex x real into a ring
            # and its N-S mirror) on the CUDA cores.  frac = roofline time / measured time
            gen, con = 2.0 * samples * NH, 8.0 * pairs * NH * B
            t_roof = (gen / ((tf32x3 if a.form == "tf32" else fp32) * 1e12) + con / (fp32 * 1e12)) * 1e3
            t_meas = sms / max(ex, 1)
            fl = (gen + con) * ex / max(nl, 1)
            ach = fl / (per_launch_ms * 1e-3) / 1e12
            peak = (gen + con) / (t_roof * 1e-3) / 1e12
            stage_rows[name] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                "frac": t_roof / t_meas,
                                "peak_source": "measured: generation at the tcgen05 tf32 rate / 3, "
                                               "contraction at the FP32 FMA rate",
                                "ms_per_step": sms / a.steps, "launches_per_step": nl / a.steps}
        elif name in ("fft_fwd", "fft_inv"):
            # algorithmic bytes: the maps (4 npix) and the compact half spectra (8 nspec) once
            by = B * (grid.npix * 4 + nspec * 8) * ex / max(nl, 1)
            # what the current layout moves: paired extended spectra (forward), kernel-grid
            # coefficients of every ring (inverse)
            lay = B * (grid.npix * 4 + (16 * ((grid.nrings + 1) // 2) * NH if name == "fft_fwd" else 8 * grid.nrings * NH))
            ach = by / (per_launch_ms * 1e-3) / 1e9
            stage_rows[name] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                                "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                                "layout_bytes_per_step": lay, "algorithmic_bytes_per_step": B * (grid.npix * 4 + nspec * 8),
                                "peak_source": f"{pk_src} HBM copy bandwidth",
                                "ms_per_step": sms / a.steps, "launches_per_step": nl / a.steps}
        else:
            stage_rows[name] = {"ms_per_step": sms / a.steps, "launches_per_step": nl / a.steps}
    dom = max(stages, key=lambda s: stages[s][0]) if stages else None
    roof = None
    if dom and "bound" in stage_rows.get(dom, {}):
        r = stage_rows[dom]
        tr = TRAFFIC.get(dom)
        traffic = None
        if tr and tr["nmaps"] == B and tr["nside"] == a.nside and tr["sources_sha256"] == sources_digest(tr["sources"]):
            traffic = tr["bytes_per_launch"]
        roof = {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                "unit": r["unit"], "frac": r["frac"], "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": r["peak_source"]}
    launches = int(sum(nl for (_, _, nl) in stages.values()))

    # whole-step roofline: T_roof = max(bytes / HBM, sum over units of flops / unit peak), with
    # the fused byte floor (read and write the maps once) and the algorithmic flops of the ring
    # FFTs (2 x 2.5 n log2 n per ring, forward and inverse) and the contraction (8 per ring
    # pair, mode and map) at the measured FP32 FMA rate, and the coefficient generation (2 per
    # sample and mode, once per beam) at the measured tcgen05 tf32 rate / 3 (3xTF32) or FP32
    ns = a.nside
    ring_n = [4 * min(i, 4 * ns - i, ns) for i in range(1, 4 * ns)]
    fft_fl = B * sum(2 * 2.5 * n * math.log2(n) for n in ring_n)
    con_fl = 8.0 * pairs * NH * B
    gen_fl = 2.0 * samples * NH
    t_bytes = 8.0 * grid.npix * B / (pk["hbm_gbs"] * 1e9) * 1e3
    t_fl = {"ring_ffts": fft_fl / (fp32 * 1e12) * 1e3, "contraction": con_fl / (fp32 * 1e12) * 1e3,
            "generation": gen_fl / ((tf32x3 if a.form == "tf32" else fp32) * 1e12) * 1e3}
    t_roof = max(t_bytes, sum(t_fl.values()))
    step_roof = {"t_roof_ms": t_roof, "bytes_ms": t_bytes, "flop_ms": t_fl, "frac": t_roof / ms,
                 "bound": "alu" if sum(t_fl.values()) > t_bytes else "hbm",
                 "peaks": {"hbm_gbs": pk["hbm_gbs"], "hbm_source": pk_src, **units,
                           "arith_source": "measured in this run (arkcos_measure_peak)"}}

    cpu = None
    if not a.no_cpu:
        knots = inputs.gaussian_knots(a.fwhm_arcmin * inputs.ARCMIN, gmax, a.knots)
        # a bounded sample of 10-20 s of host work: 192 equatorial output rings (3.7 s for 64
        # rings on 16 Grace cores)
        run, px, cores, desc = oracle_sample(a.nside, knots, gmax, rings_per_step=192)
        t = run()
        cpu = {"value": px / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc, "seconds": t}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if a.form == "fp32" else "tf32x3/f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "grid": "healpix", "nside": a.nside,
                       "maps_per_gpu": B, "global_maps": B * world,
                       "beams": a.beams, "form": "3xtf32-tensor-core" if a.form == "tf32" else "plain-fp32",
                       "l2": "inputs larger than L2 (maps of 3.2 GB per step at the default size)",
                       "launch_shape": tuned,
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "roofline": roof, "step_roofline": step_roof, "cpu_baseline": cpu,
            "clocks": clocks.summary(),
            "gpu_launches": launches, "stages": stage_rows, "other_form": other, **extras}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
