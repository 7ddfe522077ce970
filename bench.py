"""Benchmark of the fused two-species multirange LB step on GB300.

Workload (default): a batch of 8 Couette cells of 1024 x 1024 sites, FP32, the
paper's footnote couplings with G_AB = 0.405, walls at U = 1e-4 .. 1e-2 (8
log-spaced speeds), seeded random densities and the linear Couette start.  One
benchmark step = 100 lattice time steps of every cell (CUDA-graph chunks),
with the FP64 shear-stress/profile reductions every 10 steps.

value    MLUPS = (cells * nx * ny) * 100 * K / device time of K steps, summed over ranks
e2e      same metric through the C ABI with host buffers: per step, the fields
         from pinned host arrays (H2D, 268 MB), 100 time steps, lb_shear_stress
         and lb_get_profile (D2H), and the Herschel-Bulkley fit of the 8 points;
         pipelined (lb_stage_fields copies step k+1's fields while step k runs),
         with the one-after-another figure beside it ("serial")
roofline fused-kernel HBM roofline: algorithmic bytes (18 populations read + 18
         written per site update) / mean kernel duration from CUDA events on
         the library's stream, against the measured copy bandwidth
cpu_baseline the FP64 oracle on this host's cores, on a bounded sample

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own 8-cell batch (weak scaling, no data
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (2-species site updates/s) and % of HBM roofline at 1 GB300; flow-curve points/s"
UNIT = "MLUPS"
BYTES_PER_SITE = {"fp32": 144, "fp16": 72, "fp16sr": 72, "fp64": 288}
FALLBACK_HBM_GBS = 6800.0
# The FP64 step is bound by the FP64 pipe, not by HBM: its roofline counts the
# FP64 pipe operations one site update issues (ncu counts of the fused tiled
# kernel at tau = 1, the workload's: dfma 124, dadd 122, dmul 60 per site; each
# occupies the pipe once) against the pipe's rate, 152 SMs x 2 FP64 operations
# per clock (the nominal 1.25 TFLOP/s of FMA at the 2070 MHz maximum SM clock),
# at the SM clock sampled in the run.  The count is the tiled kernel's; for the
# generic kernel pair the line reports no FP64 roofline.
FP64_OPS_PER_SITE = 124 + 122 + 60
FP64_OPS_PER_CLOCK, N_SM, SM_MAX_MHZ = 2, 152, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--cells", type=int, default=8)
    ap.add_argument("--chunk", type=int, default=100, help="lattice time steps per benchmark step")
    ap.add_argument("--every", type=int, default=10, help="sampling interval of the FP64 reductions")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp16sr", "fp64"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "generic", "tiled"])
    ap.add_argument("--tau-b", type=float, default=0.0,
                    help="relaxation time of species B (0: tau = 1 for both, the paper's model); "
                         "a time per species runs the common-velocity variant")
    ap.add_argument("--mrt", default="",
                    help="s_e,s_eps,s_q,s_nu (e.g. 1.4,1.1,1.2,1.1): the multiple-relaxation-time collision with these rates "
                         "(a method variant; default: the paper's BGK collision)")
    ap.add_argument("--tile", default="", help="TXxTY for the tiled kernel (default: autotune)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bound of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bvp-steps", type=int, default=2000,
                    help="time steps of the batched-vs-plain flow-curve leg (64 cells of 512^2); 0 skips it")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="only time the FP64 oracle on this host: 1 thread and all cores, at the parity (64^2), "
                         "bench (1024^2) and precision-study (4096^2) cell sizes; one JSON line, no GPU")
    return ap.parse_args()


def dist_env():
    from paper_1004_5058_gb300.dist import rank_world
    return rank_world()


def mrt_rates(spec):
    """{s_e, s_eps, s_q, s_nu} from "a,b,c,d" ({} for an empty string: BGK)."""
    if not spec:
        return {}
    v = [float(x) for x in spec.split(",")]
    if len(v) != 4:
        raise SystemExit("--mrt wants four rates s_e,s_eps,s_q,s_nu")
    return dict(zip(("s_e", "s_eps", "s_q", "s_nu"), v))


def workload_cells(nx, ny, n_cells, rank, tau_b=0.0, mrt=""):
    from paper_1004_5058_gb300 import inputs as I
    speeds = I.log_spaced(1e-4, 1e-2, n_cells) if n_cells > 1 else [1e-3]
    return [I.make_cell("paper", nx=nx, ny=ny, g_ab=0.405, bc=1, u_wall=u, tau_b=tau_b, **mrt_rates(mrt))
            for u in speeds]


def workload_fields(nx, ny, cells, seed):
    from paper_1004_5058_gb300 import inputs as I
    ra, rb = I.random_fields(nx, ny, n_cells=len(cells), seed=seed)
    ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in cells], n_cells=len(cells))
    return ra, rb, ux, uy


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_digest():
    """Digest of the fused kernel's code (comments and layout removed, so that
    editing a comment does not orphan the committed DRAM counters)."""
    import re
    h = hashlib.sha256()
    for f in ("lb_tiled.cu", "lb_common.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_1004_5058_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(precision, nx, ny, n_cells, two_time=False, mrt=False):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    scaled to this workload's sites, if it was taken on the current sources.
    Cells with a relaxation time per species run the general kernel, and cells
    with multiple relaxation times the MRT kernel; each has its own entry
    ("<precision>_two_time", "<precision>_mrt"); without one the traffic is
    unknown."""
    p = os.path.join(ROOT, "profiles", "fused_step_dram.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(precision + ("_mrt" if mrt else "_two_time" if two_time else ""))
    if not e or d.get("source_digest") != source_digest():
        return None
    per_site = float(e["dram_bytes_per_launch"]) / float(e["sites_per_launch"])
    return per_site * nx * ny * n_cells


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(args):
    """The workload keys both arms report (the GPU arm adds its kernel and tile)."""
    n_cells, nx, ny, chunk = args.cells, args.nx, args.ny, args.chunk
    bytes_pop = 2 * n_cells * nx * ny * BYTES_PER_SITE[args.precision] / 2
    return {"workload": "couette batch: %d cells of %dx%d, %s, %d time steps per step, FP64 "
                        "reductions every %d" % (n_cells, nx, ny, args.precision.upper(), chunk, args.every),
            "cells": n_cells, "nx": nx, "ny": ny, "lattice_steps_per_step": chunk,
            "sampling_every": args.every, "precision": args.precision,
            "couplings": "paper footnote, G_AB=0.405", "u_wall": "1e-4..1e-2 log",
            "tau": "1 (both species)" if args.tau_b == 0 else "A 1, B %g (common-velocity variant)" % args.tau_b,
            "collision": ("BGK (the paper's)" if not args.mrt else
                          "multiple relaxation times s_e,s_eps,s_q,s_nu = %s (method variant)" % args.mrt),
            "l2": "inputs larger than L2 (%.2f GB populations, ping-pong)" % (bytes_pop / 1e9)}


def cpu_baseline(args, seconds):
    """The FP64 oracle, as it stands, on this host's cores: one cell of the
    workload, as many time steps as fit in about `seconds`."""
    from oracle import lb as orc
    cells = workload_cells(args.nx, args.ny, args.cells, 0, args.tau_b, args.mrt)
    cell = cells[len(cells) // 2]
    ra, rb, ux, uy = workload_fields(args.nx, args.ny, [cell], seed=1004)
    run = orc.Run(cell, ra[0], rb[0], ux[0], uy[0])
    run.set_sampling(0, args.every)
    cores = orc.max_threads()
    t0 = time.perf_counter()
    steps = 0
    while True:
        run.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 100000:
            break
    mlups = args.nx * args.ny * steps / el / 1e6
    return {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 cell of %dx%d (Couette U=%.3g), %d FP64 time steps in %.1f s" %
                      (args.nx, args.ny, cell.u_wall, steps, el)}


def cpu_sweep():
    """The CPU baseline leg at several sizes: the FP64 oracle, as it stands, on
    one thread and on all host cores.  Each entry runs whole time steps for a
    bounded time (a 4096^2 step takes seconds); MLUPS are per measured step, so
    longer runs are extrapolated linearly (the cost per step is constant)."""
    from oracle import lb as orc
    from paper_1004_5058_gb300 import inputs as I
    cores = orc.max_threads()
    out = {"kind": "oracle", "unit": UNIT, "host_cores": cores, "runs": []}
    for n, bc, budget in ((64, 0, 5.0), (1024, 1, 12.0), (4096, 1, 25.0)):
        cell = I.make_cell("paper", nx=n, ny=n, g_ab=0.405, bc=bc, u_wall=1e-3 if bc else 0.0)
        ra, rb = I.random_fields(n, n, seed=1004)
        ux, uy = I.couette_velocity(n, n, [1e-3]) if bc else (None, None)
        for threads in (1, cores):
            run = orc.Run(cell, ra[0], rb[0], None if ux is None else ux[0], None if uy is None else uy[0],
                          threads=threads)
            run.step(1)  # first touch of the arrays
            t0 = time.perf_counter()
            steps = 0
            while True:
                run.step(1)
                steps += 1
                el = time.perf_counter() - t0
                if el >= budget / 2 or steps >= 1000:
                    break
            out["runs"].append({"n": n, "bc": "couette" if bc else "periodic", "threads": threads, "steps": steps,
                                "seconds": el, "mlups": n * n * steps / el / 1e6})
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    K, W = args.steps, args.warmup
    per_step = max(1.0, min(args.cpu_seconds, 60.0 / max(1, K + W)))
    from oracle import lb as orc
    cells = workload_cells(args.nx, args.ny, args.cells, 0, args.tau_b, args.mrt)
    cell = cells[len(cells) // 2]
    ra, rb, ux, uy = workload_fields(args.nx, args.ny, [cell], seed=1004)
    run = orc.Run(cell, ra[0], rb[0], ux[0], uy[0])
    run.set_sampling(0, args.every)

    def one_step():
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < per_step:
            run.step(1)
            n += 1
        return n, time.perf_counter() - t0

    for _ in range(W):
        one_step()
    tot_n, tot_t = 0, 0.0
    for _ in range(K):
        n, t = one_step()
        tot_n += n
        tot_t += t
    mlups = args.nx * args.ny * tot_n / tot_t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
        "warmup": W, "ms_per_step": 1e3 * tot_t / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args),
                       timed="the FP64 oracle on the host cores: 1 cell of %dx%d (Couette U=%.3g) of this workload, "
                             "FP64" % (args.nx, args.ny, cell.u_wall),
                       timed_cells=1, timed_precision="fp64", timed_impl="oracle (CPU)"),
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
                         "sample": "1 cell of %dx%d, %d FP64 time steps in %.1f s over %d timed steps" %
                                   (args.nx, args.ny, tot_n, tot_t, K)},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_vs_plain(args, torch, Lattice, hb_fit):
    """The batched flow-curve sweep against the plain single-cell runs, on the
    64-cell shape of the batched flow curve: 64 Couette cells of 512 x 512 (16
    wall speeds 1e-5 .. 1e-2 log-spaced x G_AB in {0.3, 0.35, 0.405, 0.45}), FP32
    (or the bench's FP16 storage), a bounded number of steps with the second
    half sampled.  Batched: one handle, tiles from the autotuner, graph-captured
    chunks of one persistent launch per step.  Plain: the same cells one after
    another, a handle each with the library's default tile, as a caller stepping
    one cell at a time would run them.  Each side is timed from the state upload
    (lb_init_fields) to the read-back of sigma and S (handle creation and
    autotuning excluded): device time of the steps (CUDA events) and wall time of
    the whole sweep; points/s = flow-curve points (cells) per wall second at this
    step count.  sigma_max_rel_diff: the largest relative difference of the
    cells' sigma_xy between the two (both are parity-checked against the FP64
    oracle in the tests)."""
    from paper_1004_5058_gb300 import inputs as I
    L, steps, every = 512, args.bvp_steps, 20
    speeds = I.log_spaced(1e-5, 1e-2, 16)
    g_abs = (0.3, 0.35, 0.405, 0.45)
    cells = [I.make_cell("paper", nx=L, ny=L, g_ab=g, bc=1, u_wall=u) for g in g_abs for u in speeds]
    n = len(cells)
    ra, rb = I.random_fields(L, L, n_cells=n, seed=2010)
    ux, uy = I.couette_velocity(L, L, [c.u_wall for c in cells], n_cells=n)

    def sweep(lat, sl):
        st = torch.cuda.ExternalStream(lat.stream_ptr)
        lat.init_fields(ra[sl], rb[sl], ux[sl], uy[sl]).set_sampling(steps // 2, every)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        lat.step(steps)
        b.record(st)
        sig, S, _ = lat.shear_stress()
        return sig, S, a.elapsed_time(b) * 1e-3

    cache_dir = os.path.join(ROOT, "paper_1004_5058_gb300", "_build")
    cache = os.path.join(cache_dir, "autotune_cache.txt") if os.path.isdir(cache_dir) else None
    with Lattice(cells, args.precision) as lat:
        lat.init_fields(ra, rb, ux, uy)
        lat.autotune(cache)
        kern_b = lat.kernel()
        sweep(lat, slice(0, n))  # the graphs of this step pattern, untimed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sig_b, S_b, dev_b = sweep(lat, slice(0, n))
        wall_b = time.perf_counter() - t0
    lats = [Lattice([c], args.precision) for c in cells]
    try:
        kern_p = lats[0].kernel()
        sig_p, S_p, dev_p = np.empty(n), np.empty(n), 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, lp in enumerate(lats):
            s_, r_, d_ = sweep(lp, slice(c, c + 1))
            sig_p[c], S_p[c], dev_p = s_[0], r_[0], dev_p + d_
        wall_p = time.perf_counter() - t0
    finally:
        for lp in lats:
            lp.close()
    sites = n * L * L
    rel = np.abs(sig_b - sig_p) / np.maximum(np.abs(sig_p), 1e-300)
    fits = {}
    for k, g in enumerate(g_abs):
        sl = slice(16 * k, 16 * (k + 1))
        ok = np.isfinite(S_b[sl]) & (S_b[sl] > 0) & np.isfinite(sig_b[sl])
        fits[str(g)] = hb_fit(S_b[sl][ok], sig_b[sl][ok]) if ok.sum() >= 3 else None
    return {
        "workload": "64 Couette cells of 512x512: 16 wall speeds 1e-5..1e-2 x G_AB {0.3,0.35,0.405,0.45}, "
                    "%s, %d time steps, second half sampled every %d" % (args.precision.upper(), steps, every),
        "cells": n, "steps": steps,
        "batched": {"mlups": sites * steps / dev_b / 1e6, "wall_s": wall_b, "points_per_s": n / wall_b,
                    "kernel": list(kern_b)},
        "plain": {"mlups": sites * steps / dev_p / 1e6, "wall_s": wall_p, "points_per_s": n / wall_p,
                  "kernel": list(kern_p)},
        "speedup_wall": wall_p / wall_b, "speedup_device": dev_p / dev_b,
        "sigma_max_rel_diff": float(np.max(rel)), "sigma_bitwise_equal": bool(np.array_equal(sig_b, sig_p)),
        "hb_fit_batched": fits,
        "_wall_batched": wall_b,
    }


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import __graft_entry__ as g
    g.build()
    from paper_1004_5058_gb300 import Lattice, hb_fit
    from paper_1004_5058_gb300.dist import max_over_ranks

    nx, ny, n_cells, chunk = args.nx, args.ny, args.cells, args.chunk
    cells = workload_cells(nx, ny, n_cells, rank, args.tau_b, args.mrt)
    ra, rb, ux, uy = workload_fields(nx, ny, cells, seed=1004 + rank)
    lat = Lattice(cells, args.precision)
    lat.init_fields(ra, rb, ux, uy)
    if args.kernel != "auto" or args.tile:
        tx, ty = (int(v) for v in args.tile.split("x")) if args.tile else (0, 0)
        lat.set_kernel(args.kernel if args.kernel != "auto" else "tiled", tx, ty)
    else:
        cache_dir = os.path.join(ROOT, "paper_1004_5058_gb300", "_build")  # the library's build folder
        lat.autotune(os.path.join(cache_dir, "autotune_cache.txt") if os.path.isdir(cache_dir) else None)
    kernel, tx, ty = lat.kernel()
    shape = lat.launch_shape()
    launch_shape = None if shape is None else dict(zip(("ctas", "ctas_sampled", "threads", "smem_bytes"), shape))
    stream = torch.cuda.ExternalStream(lat.stream_ptr)
    lat.set_sampling(0, args.every)

    def barrier():
        if pg:
            pg.barrier()

    # warm-up
    for _ in range(args.warmup):
        lat.step(chunk)
    lat.sync()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = lat.kernel_launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lat.step(chunk)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    launches = lat.kernel_launches - launches0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = max_over_ranks(ms, device="cuda")  # the job takes as long as its slowest rank
    sites = nx * ny * n_cells
    value = sites * chunk * args.steps * world / (ms * 1e-3) / 1e6
    sigma, S, Sb = lat.shear_stress()

    # roofline: fused kernel alone (sampling off), CUDA events on the same stream;
    # the same number of steps is run once untimed first, so the CUDA graphs of
    # the timed call exist already (capture is host work that would idle the GPU)
    def timed_steps(n):
        lat.step(n)
        lat.sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        l0 = lat.kernel_launches
        a.record(stream)
        lat.step(n)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) * 1e-3 / n, (lat.kernel_launches - l0) / n

    lat.set_sampling(0, 0)
    n_roof = max(50, min(400, int(2e9 / (sites * BYTES_PER_SITE[args.precision]) * 20)))
    t_plain, kernels_per_step = timed_steps(n_roof)
    t_launch = t_plain / kernels_per_step
    # sampled steps alone (every step sampled: the SAMPLE variant of the fused
    # kernel plus the FP64 accumulation of its partial sums)
    lat.set_sampling(0, 1)
    n_samp = max(20, n_roof // 4)
    t_sampled, launches_sampled = timed_steps(n_samp)
    n_sampled_per_step = chunk // args.every if args.every > 0 else 0
    predicted_ms = 1e3 * ((chunk - n_sampled_per_step) * t_plain + n_sampled_per_step * t_sampled)
    alg_bytes = BYTES_PER_SITE[args.precision] * sites
    peak, peak_kind = peaks()
    achieved = alg_bytes / (t_launch if kernels_per_step == 1 else t_launch * kernels_per_step) / 1e9
    traffic = (committed_traffic(args.precision, nx, ny, n_cells, two_time=args.tau_b not in (0.0, 1.0),
                                 mrt=bool(args.mrt)) if kernel == "tiled" else None)

    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "%s copy bandwidth" % peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes, "mean_launch_ms": t_launch * 1e3,
                "bytes_per_site_update": BYTES_PER_SITE[args.precision],
                "launches_timed": n_roof,
                # the timed region reconciled from separately timed plain and sampled steps
                "sampled_step_ms": t_sampled * 1e3, "sampled_step_launches": launches_sampled,
                "predicted_ms_per_step": predicted_ms, "measured_ms_per_step": ms / args.steps}
    if args.precision == "fp64":
        sm_mhz = (clk or {}).get("sm_mhz") or SM_MAX_MHZ
        p64 = N_SM * FP64_OPS_PER_CLOCK * sm_mhz * 1e-3
        # the op count is the BGK kernel's (the MRT one adds its correction)
        gops = FP64_OPS_PER_SITE * sites / t_plain / 1e9 if kernel == "tiled" and not args.mrt else None
        roofline = {"bound": "alu", "achieved": gops, "peak": p64, "unit": "G FP64 op/s",
                    "frac": None if gops is None else gops / p64, "kernel": kernel,
                    "traffic": traffic,
                    "peak_source": "FP64 pipe: 152 SMs x 2 ops per clock at the sampled SM clock (%.0f MHz)" % sm_mhz,
                    "fp64_ops_per_site_update": FP64_OPS_PER_SITE, "mean_launch_ms": t_launch * 1e3,
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak}}

    # end to end through the C ABI with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_ra, h_rb, h_ux, h_uy = pin(ra), pin(rb), pin(ux), pin(uy)
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        lat.init_fields(h_ra, h_rb, h_ux, h_uy)
        lat.set_sampling(chunk // 2, args.every)
        lat.step(chunk)
        s, r, _ = lat.shear_stress()
        lat.profile()
        ok = np.isfinite(r) & (r > 0)
        if ok.sum() >= 3:
            hb_fit(r[ok], s[ok])

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_serial = sites * chunk * e2e_steps * world / e2e_s / 1e6

    # the same steps pipelined through the staged entry points: step k+1's fields
    # go to the device on the handle's copy stream while step k's time steps run,
    # and step k-1's Herschel-Bulkley fit runs on the host meanwhile
    def fit(res):
        s, r = res
        ok = np.isfinite(r) & (r > 0)
        if ok.sum() >= 3:
            hb_fit(r[ok], s[ok])

    def pipelined(n):
        lat.stage_fields(h_ra, h_rb, h_ux, h_uy)
        prev = None
        for k in range(n):
            lat.init_fields_staged()
            if k + 1 < n:
                lat.stage_fields(h_ra, h_rb, h_ux, h_uy)
            lat.set_sampling(chunk // 2, args.every)
            lat.step(chunk)
            if prev is not None:
                fit(prev)
            s, r, _ = lat.shear_stress()
            lat.profile()
            prev = (s, r)
        fit(prev)

    pipelined(2)
    barrier()
    t0 = time.perf_counter()
    pipelined(e2e_steps)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = sites * chunk * e2e_steps * world / e2e_s / 1e6
    h2d = 4 * sites * 8
    d2h = n_cells * 8 * 2 + n_cells * 8 * 2 + n_cells * ny * 8 + n_cells * 8 * 2

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16-storage/f32", "fp16sr": "f16-storage/f32",
                                       "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": dict(workload_config(args), kernel=kernel, tile=[tx, ty], launch=launch_shape),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "lattice_steps_per_step": chunk, "steps": e2e_steps,
                "pipelining": "step k+1's fields copied (lb_stage_fields, copy stream) during step k",
                "serial": {"value": e2e_serial,
                           "how": "lb_init_fields (synchronous copy), steps, results, fit, one after another"}},
        "gpu_launches": int(launches),
        "clocks": clk,
        "flow_curve": {"sigma_xy": [float(v) for v in sigma], "shear_rate": [float(v) for v in S]},
    }
    lat.close()
    if args.bvp_steps > 0 and args.precision in ("fp32", "fp16", "fp16sr") and args.tau_b == 0.0 and not args.mrt:
        bvp = batched_vs_plain(args, torch, Lattice, hb_fit)
        bvp_s = max_over_ranks(bvp.pop("_wall_batched"), device="cuda")
        bvp["batched"]["points_per_s_all_ranks"] = bvp["cells"] * world / bvp_s
        line["batched_vs_plain"] = bvp
        line["flow_curve_points_per_s"] = bvp["batched"]["points_per_s_all_ranks"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.cpu_sweep:
        return cpu_sweep()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
