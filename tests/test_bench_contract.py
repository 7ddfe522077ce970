"""The one-line JSON contract of bench.py: the reference arm (the FP64 oracle
on the host, no GPU) here, the GPU arm under the gpu marker."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e"}


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--nx", "64", "--ny", "64",
                  "--cells", "2", "--cpu-seconds", "0.5")
    assert BASE_KEYS <= set(d) and d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["config"]["workload"].startswith("couette batch: 2 cells of 64x64")
    # the line says what the reference arm actually times: one cell, FP64, the oracle
    assert d["config"]["timed_cells"] == 1 and d["config"]["timed_precision"] == "fp64"
    assert "oracle" in d["config"]["timed"]


def test_reference_arm_two_relaxation_times():
    """--tau-b reaches the oracle's cells and the reported configuration."""
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--nx", "32", "--ny", "32",
                  "--cells", "2", "--cpu-seconds", "0.3", "--tau-b", "0.7")
    assert d["value"] > 0 and d["config"]["tau"].startswith("A 1, B 0.7")


def test_reference_arm_under_torchrun_prints_once():
    """Launched like the multi-GPU bench (two ranks), the reference arm runs on
    rank 0 only: one JSON line, every rank exits 0."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--nx", "32", "--ny", "32",
           "--cells", "2", "--cpu-seconds", "0.3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0


@pytest.mark.gpu
def test_gpu_arm_line():
    d = run_bench("--steps", "3", "--warmup", "3", "--nx", "256", "--ny", "256", "--cells", "2", "--chunk", "20",
                  "--cpu-seconds", "0.5", "--bvp-steps", "200")
    assert BASE_KEYS <= set(d) and "impl" not in d
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["dtype"] == "f32" and d["data"] == "synthetic"
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 2 and rf["peak"] > 0
    assert abs(rf["achieved"] / rf["peak"] - rf["frac"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 4 * 2 * 256 * 256 * 8 and e["d2h_bytes_per_step"] > 0
    assert e["serial"]["value"] > 0 and e["pipelining"]
    assert d["gpu_launches"] >= 3 * 20
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert set(d["clocks"] or {}) >= {"sm_mhz", "sm_max_mhz", "reasons"} or d["clocks"] is None
    # the persistent grid the runtime gave the tiled kernel
    launch = d["config"]["launch"]
    assert launch["ctas"] > 0 and launch["ctas_sampled"] > 0 and launch["threads"] == d["config"]["tile"][0] + 32
    # plain and sampled steps timed apart, and the timed region predicted from them
    assert rf["sampled_step_ms"] > 0 and rf["predicted_ms_per_step"] > 0 and rf["measured_ms_per_step"] > 0
    # the batched flow-curve sweep against the same cells run one at a time
    bvp = d["batched_vs_plain"]
    assert bvp["cells"] == 64 and bvp["steps"] == 200
    assert bvp["batched"]["points_per_s"] > 0 and bvp["plain"]["points_per_s"] > 0
    assert bvp["sigma_max_rel_diff"] <= 1e-5  # same kernels: equal to rounding (bitwise when tiles agree)
    assert d["flow_curve_points_per_s"] == bvp["batched"]["points_per_s_all_ranks"]


def test_traffic_record_matches_the_kernel_sources():
    """The committed DRAM counters carry the digest of the fused kernel's code
    (comments and layout ignored); while it matches, the bench reports them and
    they stay within 10 % of the algorithmic bytes."""
    import importlib.util
    import re
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    rec = json.load(open(os.path.join(ROOT, "profiles", "fused_step_dram.json")))
    if rec["source_digest"] != bench.source_digest():
        # the kernel changed since the capture: the bench reports traffic null
        assert bench.committed_traffic("fp32", 1024, 1024, 8) is None
        pytest.skip("DRAM counters predate the current kernel code")
    assert {"fp32", "fp16", "fp16sr", "fp64"} <= set(rec)
    for prec in ("fp32", "fp16", "fp16sr"):
        per_site = rec[prec]["dram_bytes_per_launch"] / rec[prec]["sites_per_launch"]
        alg = {"fp32": 144, "fp16": 72, "fp16sr": 72}[prec]
        assert 0.9 * alg < per_site < 1.1 * alg  # no wasted re-reads
    assert bench.committed_traffic("fp32", 1024, 1024, 8) == rec["fp32"]["dram_bytes_per_launch"]
    # a relaxation time per species runs the general kernel: its own entry, or none
    two = bench.committed_traffic("fp32", 1024, 1024, 8, two_time=True)
    assert two == (rec["fp32_two_time"]["dram_bytes_per_launch"] if "fp32_two_time" in rec else None)
    assert bench.committed_traffic("fp64", 1024, 1024, 8, two_time=True) is None
    # the multiple-relaxation-time kernel moves the same bytes
    mrt = bench.committed_traffic("fp32", 1024, 1024, 8, mrt=True)
    assert mrt == (rec["fp32_mrt"]["dram_bytes_per_launch"] if "fp32_mrt" in rec else None)
    if mrt is not None:
        assert 0.9 * 144 < mrt / (8 * 1024 * 1024) < 1.1 * 144
