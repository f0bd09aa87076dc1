"""Benchmark: PRISM STEM simulation on one GB300 (or N independent replicas under torchrun).

A step is one pass of the whole PRISM hot path over one synthetic workload: transmission, the
compact S-matrix build (multislice of all 129 beams through 50 slices of a 1024^2 grid) and the
scan of all 200 x 200 probe positions (coefficients, window gather, beam sum, window FFT, bins).
Inputs (potential slices, probe positions) are resident in HBM when the timed region starts.

Printed (rank 0, one JSON line): probes/s of the PRISM step (value), plain GPU multislice probes/s
on a probe subset of the same workload, the end-to-end figure through the C ABI with host buffers,
the roofline of the dominant kernel, the FP64 oracle timed on the host cores (cpu_baseline), SM
clocks sampled during the timed region.  The headline region runs with no per-launch events; the
roofline's per-kernel durations come from a second run of the same steps in which every launch is
bracketed by CUDA events on the plan's stream.

``--impl reference`` times the FP64 oracle instead (the only reference implementation: the paper
ships none), on a bounded sample of the same workload, and prints the same line shape.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "STEM probes/s, PRISM vs multislice on one GB300 at ≤1e-3 rel err; p99 latency"
UNIT = "probes/s"
DET = dict(start_mrad=0.0, step_mrad=1.0, nbins=100)


def max_over_ranks(dist, ms, device):
    """The slowest rank's time (ms): a barrier-bracketed region timed on every rank, reduced with MAX
    (dist None: single process)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, ms):
    """Units per second of the whole job: every rank (a replica of the workload) processed
    units_per_rank per step for `steps` steps within `ms` (the slowest rank's time)."""
    return world * units_per_rank * steps / (ms / 1000.0)


def workload_config(w, B):
    return {
        "workload": f"amorphous carbon 50x50x100 A (25000 Z=6 atoms, seed 1), {w.nx}x{w.ny} grid, "
                    f"{w.n_slices} slices of {w.dz} A, {w.kv:.0f} kV, {w.alpha_mrad:.0f} mrad, f={w.f}, "
                    f"{w.scan_px}x{w.scan_py} probes at {w.scan_step} A, {DET['nbins']} x 1 mrad bins",
        "nx": w.nx, "ny": w.ny, "slices": w.n_slices, "f": w.f, "beams": B,
        "probes": w.scan_px * w.scan_py, "window_px": w.nx // w.downsample // w.f,
        "l2": "no flush: inputs larger than L2 (V 210 MB, S-matrix 270 MB, wave stack 1.08 GB vs 129 MB L2)",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------------ oracle timing (CPU)
def oracle_sample(w, V, budget_s=20.0):
    """Time the FP64 oracle as it stands on a bounded sample of the workload and extrapolate.

    Sample: four beams of the S-matrix build spread over the beam set (one oracle multislice of
    each plane wave through all slices; more while the budget lasts) and the oracle probe scan of a
    few hundred probes against a 129-beam S-matrix tiled from the first beam (the scan's cost does
    not depend on the values).  Returns probes/s for the whole workload.
    """
    from oracle import prism_oracle as O

    g = dict(nx=w.nx, ny=w.ny, cell_x=w.cell_x, cell_y=w.cell_y, n_slices=w.n_slices, dz=w.dz, kv=w.kv,
             f=w.f, downsample=w.downsample, aa_frac=w.aa_frac, alpha_mrad=w.alpha_mrad)
    m, n = O.beam_set(w.nx, w.ny, w.cell_x, w.cell_y, w.kv, w.f, w.alpha_mrad)
    B = len(m)
    t0 = time.perf_counter()
    trans = O.transmission(V, w.kv)
    prop = O.slice_propagators(g)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    s0 = None
    n_beam = 0
    while n_beam < 4 or (n_beam < B and time.perf_counter() - t0 < 0.6 * budget_s):
        b = (n_beam * B) // 4 if n_beam < 4 else n_beam
        pw = O.plane_wave(w.nx, w.ny, w.cell_x, w.cell_y, m[b] * w.f / w.cell_x, n[b] * w.f / w.cell_y)
        sb = O.fourier_crop_half(O.multislice(pw, trans, prop))
        s0 = sb if s0 is None else s0
        n_beam += 1
    t_beam = (time.perf_counter() - t0) / n_beam
    S = np.broadcast_to(s0, (B,) + s0.shape)
    x0, y0 = w.scan_positions()
    n_probe = 0
    t0 = time.perf_counter()
    while True:
        O.prism_scan(S, m, n, g, dict(alpha_mrad=w.alpha_mrad), DET, x0[n_probe:n_probe + 4], y0[n_probe:n_probe + 4])
        n_probe += 4
        if time.perf_counter() - t0 > max(1.0, budget_s - n_beam * t_beam - t_setup) or n_probe >= 400:
            break
    t_probe = (time.perf_counter() - t0) / n_probe
    P = w.scan_px * w.scan_py
    total = t_setup + B * t_beam + P * t_probe
    return {
        "value": P / total, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
        "sample": f"FP64 NumPy oracle: {n_beam} of {B} S-matrix beams ({w.n_slices} slices, {w.nx}^2) at {t_beam:.2f} s each, "
                  f"{n_probe} of {P} probe scans in {t_probe * n_probe:.2f} s, transmission/propagator setup "
                  f"{t_setup:.2f} s; extrapolated to the full workload ({total:.0f} s). numpy.fft single-threaded, "
                  f"BLAS contraction with the library's default threads",
        "seconds_measured": t_setup + n_beam * t_beam + t_probe * n_probe,
    }


# device code of the row and column pass kernels (the ones profiles/dram_traffic.json measures):
# the kernel templates and their helpers, the compiled launch shapes, and the parameter blocks the
# kernels read (host-only declarations in params.h do not enter the hash)
PASS_SOURCES = ("fft.cuh", "pass_kernels.cuh", "pass_default.cuh", "tc.cuh", "kernels_build.cu", "tune_shapes.cuh")
PASS_STRUCTS = ("struct Tw64", "struct RowArgs", "struct ColArgs")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1702_01904_gb300", "csrc")
    for f in PASS_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    params = open(os.path.join(csrc, "params.h")).read()
    for name in PASS_STRUCTS:
        i = params.index(name)
        h.update(params[i:params.index("};", i) + 2].encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """Bytes per launch from the committed ncu summary, if it was taken on the current sources."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("bytes_per_launch_full")


def serving_run(n_requests=60, rate=20.0, seed=5, budget_gb=48):
    """Poisson stream of simulation requests through the continuous-batching engine.

    Half the requests are small cells (16 A simple-cubic Cu, 256^2, 8 slices, f=4, 16x16 probes,
    private S-matrix each); half are region-of-interest scans (32 x 32 probes at a probe step drawn
    from 0.2-0.5 A, at a random place) of the large serving cell (102.4 A nanoparticle on carbon,
    2048^2, 100 slices, f=8, 529 beams), all served by one resident S-matrix (key 1) made before
    the stream starts.  Admission is by HBM footprint under a budget of `budget_gb`.  Returns
    latency percentiles (submission -> result in host memory) and throughput."""
    import torch

    from paper_1702_01904_gb300 import prism as PR
    from paper_1702_01904_gb300 import specimens
    from paper_1702_01904_gb300.runtime import Server

    rng = np.random.Generator(np.random.PCG64(seed))
    small = specimens.workload_small()
    Vs = torch.from_numpy(small.potential()).pin_memory()
    t_gen = time.perf_counter()
    big = specimens.workload_nanoparticle_on_carbon(n_slices=100)
    Vl = torch.from_numpy(specimens.project_potential_parallel(big.specimen, big.nx, big.ny, big.n_slices,
                                                               big.dz)).pin_memory()
    t_gen = time.perf_counter() - t_gen
    gs, gl = PR.grid_from_workload(small), PR.grid_from_workload(big)
    det = PR.make_detector(DET["start_mrad"], DET["step_mrad"], DET["nbins"])
    probe = PR.make_probe(20.0)
    xs_s, ys_s = small.scan_positions()
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    kinds = rng.random(n_requests) < 0.5
    steps = rng.choice([0.2, 0.25, 0.3, 0.4, 0.5], n_requests)
    origins = rng.uniform(0.0, big.cell_x, (n_requests, 2))
    budget = budget_gb << 30
    srv = Server(hbm_budget_bytes=budget, max_inflight=8)

    def roi(i):
        g1 = np.arange(32) * steps[i]
        yy, xx = np.meshgrid(origins[i, 1] + g1, origins[i, 0] + g1, indexing="ij")
        return xx.ravel(), yy.ravel()

    # warm the code paths and make the large cell's S-matrix resident (not part of the stream)
    t, _ = srv.submit(gs, Vs, probe, xs_s, ys_s, det)
    srv.wait(t)
    x, y = roi(0)
    t, _ = srv.submit(gl, Vl, probe, x, y, det, key=1, px=32, py=32)
    cold = srv.wait(t, timeout_s=1200.0)
    tickets = []
    probes = 0
    t0 = time.perf_counter()
    for i in range(n_requests):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        if kinds[i]:
            t, _ = srv.submit(gs, Vs, probe, xs_s, ys_s, det)
            probes += len(xs_s)
        else:
            x, y = roi(i)
            t, _ = srv.submit(gl, Vl, probe, x, y, det, key=1, px=32, py=32)
            probes += 32 * 32
        tickets.append(t)
    lat, reused = [], 0
    by_kind = {True: [], False: []}
    for k, t in zip(kinds, tickets):
        st = srv.wait(t)
        lat.append(st.total_ms)
        by_kind[bool(k)].append(st.total_ms)
        reused += st.smatrix_reused
    wall = time.perf_counter() - t0
    info = srv.stats()
    srv.close()
    lat = np.sort(np.array(lat))
    pct = lambda v, q: float(np.percentile(np.array(v), q)) if len(v) else None
    return {"requests": n_requests, "poisson_rate_per_s": rate, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat[-1]), "requests_per_s": n_requests / wall, "probes_per_s": probes / wall,
            "small_cell_p50_ms": pct(by_kind[True], 50), "small_cell_p99_ms": pct(by_kind[True], 99),
            "large_cell_p50_ms": pct(by_kind[False], 50), "large_cell_p99_ms": pct(by_kind[False], 99),
            "large_cell_first_request_ms": cold.total_ms,
            "smatrix_reused": int(reused), "peak_device_bytes": int(info.peak_bytes), "hbm_budget_bytes": budget,
            "large_cell_potential_s": t_gen,
            "mix": "50% 16 A Cu cells (256^2, 8 slices, f=4, 256 probes, own S-matrix each); 50% 32x32-probe "
                   "scans at 0.2-0.5 A steps of the 102.4 A Au-on-a-C cell (2048^2, 100 slices, f=8, 529 beams, "
                   "4.4 GB S-matrix) from one resident S-matrix made before the stream (its first request: "
                   "large_cell_first_request_ms)"}


def batch_leg(n_cells=64, runs=2, n_branches=4, autotune=True):
    """The batched workload: n_cells seeded uneven cells (seeds 100...), FP32, one captured CUDA
    graph per run (prism_batch_*).  Potentials are generated by a spawn process pool."""
    import multiprocessing as mp

    import torch

    from paper_1702_01904_gb300 import prism as PR
    from paper_1702_01904_gb300 import specimens
    from paper_1702_01904_gb300.runtime import Batch

    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        made = pool.map(specimens.batch_cell_potential, range(100, 100 + n_cells))
    gen_s = time.perf_counter() - t0
    det = PR.make_detector(DET["start_mrad"], DET["step_mrad"], DET["nbins"])
    stream = torch.cuda.Stream()
    cells, beams_slices, probes, mix, build_bytes = [], 0, 0, {}, 0
    for w, V in made:
        x0, y0 = w.scan_positions()
        cells.append(dict(grid=PR.grid_from_workload(w), V=torch.from_numpy(V).cuda(), probe=PR.make_probe(w.alpha_mrad),
                          x0=x0, y0=y0, px=w.scan_px, py=w.scan_py, det=det))
        lam = PR.prism_wavelength(w.kv)
        r = w.alpha_mrad * 1e-3 / (lam * w.f / w.cell_x)
        k = np.arange(-int(r) - 1, int(r) + 2)
        nb = int(np.count_nonzero(k[:, None] ** 2 + k[None, :] ** 2 <= r * r * (1 + 1e-12)))
        beams_slices += nb * w.n_slices
        # build passes stream the kept columns of the wave stack twice per slice (32 B per kept
        # beam-pixel) plus t_p
        fk = (2 * (int(math.ceil(w.aa_frac * w.nx / 2)) - 1) + 1) / w.nx
        build_bytes += nb * w.n_slices * w.nx * w.ny * 32 * fk + w.n_slices * w.nx * w.ny * 8
        probes += w.scan_px * w.scan_py
        key = f"{w.nx}px_f{w.f}"
        mix[key] = mix.get(key, 0) + 1
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t1 = time.perf_counter()
        b = Batch(cells, n_branches=n_branches, stream=stream, autotune=autotune, fft_radix=autotune)
        create_s = time.perf_counter() - t1
        b.run()
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(runs):
            b.run()
        e1.record(stream)
        b.sync()
        ms = e0.elapsed_time(e1) / runs
        info = b.info
        b.close()
    return {"cells": n_cells, "seeds": f"100..{99 + n_cells}", "size_mix": mix, "runs_timed": runs,
            "ms_per_run": ms, "cells_per_s": n_cells / (ms / 1000.0), "probes_per_s": probes / (ms / 1000.0),
            "beams_slices_per_s": beams_slices / (ms / 1000.0), "graph_nodes": info.graph_nodes,
            "build_pass_bytes_per_run": build_bytes,
            "build_pass_gbs_over_whole_run": build_bytes / (ms / 1000.0) / 1e9,
            "kernel_launches_per_run": info.kernel_launches, "branches": info.n_branches,
            "device_gb": info.device_bytes / 1e9, "potential_generation_s": gen_s,
            "create_s": create_s, "autotuned": autotune,
            "what": "every cell's transmission + S-matrix build + 16x16-probe scan, FP32, one cudaGraphLaunch per run"}


def ncu_case(precision="fp32", full_k=False):
    import torch

    from paper_1702_01904_gb300 import prism as PR
    from paper_1702_01904_gb300 import specimens
    from paper_1702_01904_gb300.runtime import PrismSimulation

    # FP32: 25 beams (alpha_max 9 mrad), the first 10 scan rows (2000 probes).  16-bit, or FP32
    # with full_k: the full 129-beam set, so that the scan sees the real K, and the first 52 rows
    # (10400 probes, 325 groups of 8 x 4: every resident CTA busy).  Both: 4 slices.
    half = precision != "fp32" or full_k
    w = specimens.workload_amorphous_carbon(n_slices=4, alpha_mrad=20.0 if half else 9.0)
    V = torch.from_numpy(w.potential()).cuda()
    x0, y0 = w.scan_positions()
    code = {"fp32": PR.PRISM_PRECISION_FP32, "fp16": PR.PRISM_PRECISION_FP16, "bf16": PR.PRISM_PRECISION_BF16,
            "fp16x2": PR.PRISM_PRECISION_FP16X2}[precision]
    sim = PrismSimulation(PR.grid_from_workload(w, precision=code))
    det = PR.make_detector(DET["start_mrad"], DET["step_mrad"], DET["nbins"])
    probe = PR.make_probe(w.alpha_mrad)
    rows = 52 if half else 10
    n = 200 * rows
    for _ in range(2):  # launches per pass: transmission, 4 x (row, col), row_out, [quantize], scan
        sim.build(V)
        sim.scan(probe, x0[:n], y0[:n], det, px=200, py=rows)
    sim.sync()
    print(json.dumps({"ncu_case": "ok", "precision": precision, "beams": sim.info.n_beams, "launches": sim.launches()}))
    sim.close()
    return 0


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ms-probes", type=int, default=1024, help="probes timed for the multislice baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16", "fp16x2"], default="fp32",
                    help="S-matrix storage / beam-sum arithmetic of the headline line")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-cells leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes of the passes")
    ap.add_argument("--batch-cells", type=int, default=64)
    ap.add_argument("--no-precision-leg", action="store_true",
                    help="skip timing the other precisions beside the headline one")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run the profiling case twice and exit: the same 1024^2 a-C grid, 4 slices, "
                         "alpha_max 9 mrad (25 beams, 200 MB wave stack), 2000 probes")
    ap.add_argument("--ncu-full-k", action="store_true",
                    help="with --ncu-case: all 129 beams and 10400 probes in every precision")
    args = ap.parse_args()
    if args.ncu_case:
        return ncu_case(args.precision, args.ncu_full_k)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1702_01904_gb300 import specimens

    if args.impl == "reference":
        if rank != 0:
            return 0
        w = specimens.workload_amorphous_carbon()
        V = w.potential()
        steps = []
        last = None
        for i in range(args.warmup + args.steps):
            r = oracle_sample(w, V, budget_s=8.0 if args.steps > 2 else 15.0)
            if i >= args.warmup:
                steps.append(r)
            last = r
        val = statistics.median([r["value"] for r in steps]) if steps else last["value"]
        P = w.scan_px * w.scan_py
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * P / val,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": workload_config(w, 129),
               "cpu_baseline": {"value": val, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                                "sample": last["sample"]},
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return 0

    import torch

    from paper_1702_01904_gb300 import build as B
    from paper_1702_01904_gb300 import prism as PR
    from paper_1702_01904_gb300.runtime import PrismSimulation, multislice

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    B.build()  # no-op once built
    dev = torch.cuda.current_device()

    w = specimens.workload_amorphous_carbon()
    V_host = torch.from_numpy(w.potential())
    V = V_host.cuda()
    x0, y0 = w.scan_positions()
    P = len(x0)
    PREC = {"fp32": PR.PRISM_PRECISION_FP32, "fp16": PR.PRISM_PRECISION_FP16, "bf16": PR.PRISM_PRECISION_BF16,
            "fp16x2": PR.PRISM_PRECISION_FP16X2}
    grid = PR.grid_from_workload(w, precision=PREC[args.precision])
    grid32 = PR.grid_from_workload(w)
    det = PR.make_detector(DET["start_mrad"], DET["step_mrad"], DET["nbins"])
    probe = PR.make_probe(w.alpha_mrad)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        sim = PrismSimulation(grid, 0, stream)
        Bn = sim.info.n_beams
        tune = None if args.no_autotune else sim.autotune(fft_radix=True)
        out = torch.empty((P, DET["nbins"]), dtype=torch.float32, device="cuda")

        def step():
            sim.build(V)
            sim.scan(probe, x0, y0, det, out=out, px=w.scan_px, py=w.scan_py)

        for _ in range(args.warmup):
            step()
        if not args.no_autotune:
            # the scan's contraction tile shape, timed on this scan (every shape writes the same stack)
            sim.autotune_scan(probe, x0, y0, det, out=out, px=w.scan_px, py=w.scan_py)
            tune = sim.tune_result()
        stream.synchronize()
        sim.reset_stats()
        sim.set_profiling(False)  # the headline region runs without per-launch events
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        clocks = ClockSampler(gpu_smi_id(torch, dev))
        clocks.start()
        time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = clocks.stop()
        total_ms = evs[0].elapsed_time(evs[-1])
        per_step = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
        launches = sim.launches()
        total_ms = max_over_ranks(dist, total_ms, "cuda")
        # per-kernel durations for the roofline: the same K steps again, each launch bracketed by
        # CUDA events on the plan's stream (this region is not the headline)
        sim.reset_stats()
        sim.set_profiling(True)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            step()
        p1.record(stream)
        stream.synchronize()
        profiled_ms_per_step = p0.elapsed_time(p1) / args.steps
        sim.set_profiling(False)
        stats = sim.kernel_stats()

        # end to end through the C ABI with host buffers (pinned), copies inside the timed region
        V_pin = V_host.pin_memory()
        out_pin = torch.empty((P, DET["nbins"]), dtype=torch.float32).pin_memory()

        def step_host():
            sim.build_host(V_pin)
            sim.scan_host(probe, x0, y0, det, out_pin, px=w.scan_px, py=w.scan_py)
            sim.sync()

        step_host()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t_e2e0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            step_host()
        e1.record(stream)
        stream.synchronize()
        e2e_ms = (time.perf_counter() - t_e2e0) * 1000.0
        e2e_ms = max_over_ranks(dist, e2e_ms, "cuda")
        h2d = V_host.numel() * 4 + P * 16
        d2h = P * DET["nbins"] * 4

        # multislice baseline on a probe subset of the same workload
        nms = min(args.ms_probes, P)
        sel = np.linspace(0, P - 1, nms).astype(np.int64)
        ms_out = torch.empty((nms, DET["nbins"]), dtype=torch.float32, device="cuda")
        multislice(grid32, V, probe, x0[sel][:8], y0[sel][:8], det, stream=stream, out=ms_out[:8])
        stream.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        multislice(grid32, V, probe, x0[sel], y0[sel], det, stream=stream, out=ms_out, scratch_bytes=2 << 30)
        m1.record(stream)
        stream.synchronize()
        ms_ms = m0.elapsed_time(m1)

        # the other precisions on the same workload: step time, scan time, and the deviation of
        # every detector image from this run's headline output
        prec_leg = {}
        if rank == 0 and not args.no_precision_leg:
            ref_out = out.cpu().numpy().astype(np.float64)
            for name in ("fp32", "fp16", "bf16", "fp16x2"):
                if name == args.precision:
                    continue
                s2 = PrismSimulation(PR.grid_from_workload(w, precision=PREC[name]), 0, stream)
                o2 = torch.empty_like(out)
                if not args.no_autotune:
                    s2.autotune(fft_radix=True)

                def step2():
                    s2.build(V)
                    s2.scan(probe, x0, y0, det, out=o2, px=w.scan_px, py=w.scan_py)

                for _ in range(2):
                    step2()
                tune2 = None
                if not args.no_autotune:
                    # the scan's shape: contraction tiles (FP32) or the tensor-core ring (16-bit)
                    s2.autotune_scan(probe, x0, y0, det, out=o2, px=w.scan_px, py=w.scan_py)
                    tune2 = {k: v["chosen"] for k, v in s2.tune_result().items()}
                stream.synchronize()
                s2.reset_stats()
                s2.set_profiling(True)
                q0 = torch.cuda.Event(enable_timing=True)
                q1 = torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                for _ in range(args.steps):
                    step2()
                q1.record(stream)
                stream.synchronize()
                st2 = s2.kernel_stats()
                t2 = q0.elapsed_time(q1) / args.steps
                o2n = o2.cpu().numpy().astype(np.float64)
                mean = ref_out.mean(0)
                dev = {}
                for floor in (1e-3, 1e-5):
                    sel2 = mean >= floor
                    e = np.linalg.norm(o2n[:, sel2] - ref_out[:, sel2], axis=0) / np.linalg.norm(ref_out[:, sel2], axis=0)
                    dev[f"images_mean_ge_{floor:g}"] = {"max_rel_l2": float(e.max()), "median_rel_l2": float(np.median(e)),
                                                        "images": int(sel2.sum())}
                scan2 = st2["scan"][1] / max(st2["scan"][0], 1)
                prec_leg[name] = {"value": P / (t2 / 1000.0), "unit": UNIT, "ms_per_step": t2, "scan_ms": scan2,
                                  "build_ms": t2 - scan2, "smatrix_bytes": PR.prism_plan_smatrix_bytes(s2.plan),
                                  "deviation_from_headline": dev, "autotune": tune2}
                s2.close()
        sim.close()

    value = whole_job_rate(world, P, args.steps, total_ms)
    ms_probes_s = nms / (ms_ms / 1000.0)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean event time per launch
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    hbm_peak = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    px = w.nx * w.ny
    # kept fraction of the mixed-domain wave: the propagator's anti-aliasing aperture zeroes every
    # column |kx| >= K+1 (K = ceil(aa_frac nx / 2) - 1 on a square cell), and the passes neither
    # read nor write those columns
    K = int(math.ceil(w.aa_frac * w.nx / 2)) - 1
    fk = (2 * K + 1) / w.nx
    # per-launch algorithmic bytes: the kept part of the wave stack read + written (8 B per complex64
    # pixel each way) for all beams, plus the slice's transmission function for the row pass
    alg = {
        "row": 2 * Bn * px * 8 * fk + px * 8,
        "col": 2 * Bn * px * 8 * fk,
        # first slice: the row transform of t_0 (read t_0, write every column), then the shifted
        # gather that writes the kept part of every beam's rows (reading the transform once)
        "row_plane": 2 * px * 8,
        "plane": Bn * px * 8 * fk + px * 8,
        "row_out": Bn * (px // 2) * 8 * fk + Bn * (px // 4) * 8,
        "transmission": w.n_slices * px * (4 + 8),
        # 16-bit mode: FP32 S of the batch read twice (scale, convert), 16-bit pixel-major S written
        "quantize": 2 * Bn * (px // 4) * 8 + (px // 4) * 2 * ((Bn + 7) // 8 * 8) * 2,
    }
    # FFT flops per launch: a row pass does an inverse and a forward length-nx transform per row of
    # every beam plus the t_p multiply (6 flops per element); a column pass the same per kept column
    # with the propagator multiply
    fl = lambda n: 5.0 * n * math.log2(n)
    fft_flops = {
        "row": Bn * w.ny * (2 * fl(w.nx) + 6.0 * w.nx),
        "col": Bn * (2 * K + 1) * (2 * fl(w.ny) + 6.0 * w.ny),
    }
    rows = {}
    for name, (n_l, t_ms) in stats.items():
        if n_l == 0:
            continue
        rows[name] = {"launches": n_l, "total_ms": t_ms, "mean_ms": t_ms / n_l}
    dominant = max(rows, key=lambda k: rows[k]["total_ms"])
    roof_all = {}
    for name, r in rows.items():
        if name in alg:
            gbs = alg[name] / (r["mean_ms"] / 1000.0) / 1e9
            roof_all[name] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                              "frac": gbs / hbm_peak, "bytes_per_launch": alg[name], **r}
            if name in fft_flops:
                # the same launch against the FP32 FFT-flop roofline (5 N log2 N per length-N transform)
                clk_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
                fp32_peak = 152 * 128 * 2 * clk_mhz * 1e6 / 1e12
                tf = fft_flops[name] / (r["mean_ms"] / 1000.0) / 1e12
                roof_all[name].update({"fft_tflops": tf, "fft_peak_tflops": fp32_peak, "fft_frac": tf / fp32_peak,
                                       "fft_flops_per_launch": fft_flops[name]})
        elif name == "scan" and args.precision != "fp32":
            # beam sum on the tensor cores: 8 real flops per complex MAC, against the measured dense
            # 16-bit rate (sustained: the scan runs inside a seconds-long loop of steps)
            nw = w.nx // w.downsample // w.f
            flops = P * 8.0 * Bn * nw * nw
            peak_tf = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0
            tf = flops / (r["mean_ms"] / 1000.0) / 1e12
            roof_all[name] = {"bound": "tensor", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                              "frac": tf / peak_tf, "flops_per_launch": flops, **r}
        elif name == "scan":
            # ALU-bound: 8 flops per complex MAC of the beam sum (a7) + window FFTs
            nw = w.nx // w.downsample // w.f
            flops = P * (8.0 * Bn * nw * nw + 2 * 5.0 * nw * nw * math.log2(nw))
            clk_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
            peak_tf = 152 * 128 * 2 * clk_mhz * 1e6 / 1e12
            tf = flops / (r["mean_ms"] / 1000.0) / 1e12
            roof_all[name] = {"bound": "alu", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                              "frac": tf / peak_tf, "flops_per_launch": flops, **r}
    dom = dominant if dominant in roof_all else max(roof_all, key=lambda k: roof_all[k]["total_ms"])
    rd = roof_all[dom]
    roofline = {"bound": rd["bound"], "achieved": rd["achieved"], "peak": rd["peak"], "unit": rd["unit"],
                "frac": rd["frac"], "traffic": ncu_traffic(dom), "kernel": dom,
                "durations": f"per-launch CUDA events on the plan's stream over a second run of the {args.steps} "
                             f"timed steps ({profiled_ms_per_step:.3f} ms per step with the events, "
                             f"{total_ms / args.steps:.3f} ms in the headline region without them)",
                "peak_source": f"{peak_note} ({'MEASURED_PEAKS.json hbm_gbs' if rd['unit'] == 'GB/s' else ('MEASURED_PEAKS.json bf16 sustained' if rd['bound'] == 'tensor' else '152 SMs x 128 FP32 lanes x 2 x median SM clock')})"}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_run()

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_leg(args.batch_cells, autotune=not args.no_autotune)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, V_host.numpy(), budget_s=20.0)
        cpu.pop("seconds_measured", None)

    if rank == 0:
        build_ms = sum(rows[k]["total_ms"] for k in rows if k != "scan") / args.steps
        scan_ms = rows.get("scan", {}).get("total_ms", 0.0) / args.steps
        lat = sorted(per_step)
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16 S / f32 accumulate", "bf16": "bf16 S / f32 accumulate",
                      "fp16x2": "f16 value + f16 remainder S / f32 accumulate"}[args.precision],
            "data": "synthetic (seeded amorphous-carbon phantom; the paper's Pt/a-C coordinates are not available)",
            "config": {**workload_config(w, Bn), "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": {"value": whole_job_rate(world, P, args.steps, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": "prism_build_smatrix_host + prism_scan_run_host, pinned host buffers, wall clock"},
            "gpu_launches": launches,
            "roofline": roofline,
            "roofline_all": roof_all,
            "cpu_baseline": cpu,
            "precision": {"headline": args.precision, "others": prec_leg,
                          "note": "16-bit modes store S in FP16/BF16 with per-beam power-of-two scales and run the beam "
                                  "sum on tcgen05 tensor cores (FP32 accumulation); their error against the FP64 oracle "
                                  "per detector image is gated in tests/test_gpu_precision.py"},
            "multislice": {"probes_per_s": ms_probes_s, "probes_timed": nms, "ms": ms_ms,
                           "speedup_prism_vs_multislice": value / world / ms_probes_s},
            "beams_slices_per_s": Bn * w.n_slices / (build_ms / 1000.0),
            "phase_ms_per_step": {"s_matrix_build": build_ms, "scan": scan_ms},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                           "what": "one whole step (S-matrix build + 40000-probe scan), device time"},
            "serving": serving,
            "batch": batch,
            "autotune": tune,
            "clocks": clk,
        }
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
