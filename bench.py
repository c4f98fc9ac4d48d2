"""Benchmark: KL nearest-neighbour descent build on one GB300.

Workload (one step = one whole build: precompute, initial graph, rounds to the
statistical stop): n = 1,000,000 Dirichlet(1) points on the 20-simplex
(21 FP32 coordinates), K = 20, seed 1, mixed form (FP32 CUDA-core filter with
a rigorous error bound, FP64 re-score; the graph equals the FP64 form's).

Metric: KL comparator evaluations per second, where the evaluations of a
build are n*K (initial graph) + rounds * n*(K + 2K^2) (the candidate multiset
of Sec. 3.1 / Sec. 4.4 per round).  The FP64 form is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (test infrastructure, never the product
path) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_00517_gb300.datagen import dirichlet_points  # noqa: E402

N, M, K, SEED = 1_000_000, 21, 20, 1
METRIC = "KNN-descent build s & KL evals/s, n=1e6 d=20 K=20: mixed vs FP64, % roofline"
UNIT = "KL evals/s"
WORKLOAD = "KL K-NN descent build to the statistical stop, n=1e6 Dirichlet(1) points, d=20 (21 FP32 coords), K=20, seed 1"
REF_ROWS = 100_000  # rows of round 1 the oracle computes per reference step


def evals_of(n, k, rounds):
    return n * k + rounds * n * (k + 2 * k * k)


# ---------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_gpu{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- roofline inputs
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def join_traffic_per_launch():
    """DRAM bytes per join launch from the committed ncu summary, if it was taken
    on the current join source (sha256 recorded in the summary); else None."""
    src = os.path.join(ROOT, "paper_2202_00517_gb300", "csrc", "join.cu")
    prof = os.path.join(ROOT, "profiles", "join_mixed_n1e6_m21_K20.md")
    if not os.path.exists(prof):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    text = open(prof).read()
    m_sha = re.search(r"join\.cu sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram bytes per full-size launch:\s*([0-9.eE+]+)", text)
    if not (m_sha and m_b) or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


# ---------------------------------------------------------------------------- reference arm
def cpu_reference_step(pts64, g0i):
    """One bounded oracle sample: round 1 of the workload for rows [0, REF_ROWS),
    starting from the oracle's own initial graph.  Returns (evaluations, seconds)."""
    import oracle
    t0 = time.perf_counter()
    _, _, _, _, props = oracle.round_(pts64, g0i, 0, REF_ROWS)
    dt = time.perf_counter() - t0
    return props, dt


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    pts64 = dirichlet_points(N, M, SEED, np.float32).astype(np.float64)
    g0i, _ = oracle.init_graph(pts64, K, SEED)
    for _ in range(args.warmup):
        cpu_reference_step(pts64, g0i)
    ev, sec = 0, 0.0
    for _ in range(args.steps):
        e, s = cpu_reference_step(pts64, g0i)
        ev += e
        sec += s
    value = ev / sec
    cores = oracle.num_threads()
    sample = (f"oracle round 1 (from its own initial graph) for rows [0, {REF_ROWS}) of the n=1e6 workload "
              "per step; setup (log table, co-friend lists over all n) included")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "m": M, "K": K, "seed": SEED,
                                            "form": "CPU oracle, FP64", "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_2202_00517_gb300 as knnd

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    dev = torch.device("cuda", local)
    pts_host = torch.from_numpy(dirichlet_points(N, M, SEED, np.float32))
    pts = pts_host.to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def run_form(prec, steps, warmup, clocks=None):
        h = knnd.Handle(N, M, K, dtype="f32", precision=prec, timing=True)
        idx, key, flag = h.new_graph(dev)
        for _ in range(warmup):
            out = h.build(pts, SEED, idx, key, flag)
        h.reset_stats()
        torch.cuda.synchronize()
        barrier()
        if clocks:
            clocks.start()
        ms_total, ev_total, infos = 0.0, 0, []
        t_wall = time.perf_counter()
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = h.build(pts, SEED, idx, key, flag)
            e1.record(stream)
            e1.synchronize()
            ms_total += e0.elapsed_time(e1)
            ev_total += evals_of(N, K, out["rounds"])
            infos.append(out)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t_wall
        clk = clocks.stop() if clocks else None
        st = h.stats()
        h.close()
        return {"ms": ms_total, "evals": ev_total, "infos": infos, "stats": st, "wall": wall, "clocks": clk}

    clocks = Clocks(local)
    mixed = run_form("mixed", args.steps, args.warmup, clocks)
    fp64 = run_form("fp64", args.fp64_steps, 1)

    # end to end through the public API from pinned host memory (H2D points, D2H idx+key)
    h = knnd.Handle(N, M, K, dtype="f32", precision="mixed")
    ph = pts_host.pin_memory()
    idx_h = torch.empty((N, K), dtype=torch.int32, pin_memory=True)
    key_h = torch.empty((N, K), dtype=torch.float64, pin_memory=True)
    h.build_host(ph, SEED, idx_h, key_h)
    e2e_sec, e2e_ev = 0.0, 0
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = h.build_host(ph, SEED, idx_h, key_h)
        e2e_sec += time.perf_counter() - t0
        e2e_ev += evals_of(N, K, out["rounds"])
    h.close()

    # max over ranks of the device time
    t = torch.tensor([mixed["ms"], fp64["ms"], e2e_sec], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mixed_ms, fp64_ms, e2e_max = t.tolist()

    if rank == 0:
        info = mixed["infos"][-1]
        st = mixed["stats"]
        steps = args.steps
        value = world * mixed["evals"] / (mixed_ms / 1e3)
        # dominant kernel: the join (mixed form), FP32 FMA pipe bound
        join_ms = st["phase_ms"]["join"]
        join_n = max(1, st["phase_count"]["join"])
        join_avg_s = join_ms / join_n / 1e3
        flops_per_launch = 2.0 * M * N * K * (2 * K + 1)
        peaks, peak_kind = measured_peaks()
        clk = mixed["clocks"] or {}
        sm_mhz = 2070.0
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
        achieved = flops_per_launch / join_avg_s / 1e12
        traffic = join_traffic_per_launch()
        phase_share = {p: (st["phase_ms"][p] / max(1e-9, sum(st["phase_ms"].values()))) for p in st["phase_ms"]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": mixed_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32+fp64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "m": M, "K": K, "seed": SEED,
                       "form": "mixed: FP32 CUDA-core join filter + FP64 re-score (graph == FP64 form)",
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "build_s_mixed": mixed_ms / steps / 1e3,
            "build_s_fp64": fp64_ms / max(1, args.fp64_steps) / 1e3,
            "evals_per_s_fp64": world * fp64["evals"] / (fp64_ms / 1e3),
            "speedup_mixed_vs_fp64": (fp64_ms / max(1, args.fp64_steps)) / (mixed_ms / steps),
            "rounds": info["rounds"], "updates": info["updates"], "fcc_hits": info["fcc_hits"],
            "rescored_per_build": info["rescored"], "merge_fallback_rows": info["merge_fallbacks"],
            "phase_ms_per_build": {p: st["phase_ms"][p] / steps for p in st["phase_ms"]},
            "phase_share": phase_share,
            "roofline": {"kernel": "join_mixed_kernel<24,1>", "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": traffic,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (max SM clock)",
                         "flops_per_launch": flops_per_launch, "avg_launch_ms": join_avg_s * 1e3,
                         "launches_timed": join_n,
                         "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_kind": peak_kind},
            "e2e": {"value": world * e2e_ev / e2e_max, "unit": UNIT,
                    "h2d_bytes_per_step": N * M * 4, "d2h_bytes_per_step": N * K * (4 + 8)},
            "gpu_launches": st["kernel_launches"],
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            import oracle
            pts64 = pts_host.numpy().astype(np.float64)
            g0i, _ = oracle.init_graph(pts64, K, SEED)
            e, s = cpu_reference_step(pts64, g0i)
            line["cpu_baseline"] = {
                "value": e / s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": (f"oracle round 1 for rows [0, {REF_ROWS}) of the n=1e6 workload from its own initial "
                           f"graph ({e} evaluations in {s:.2f} s, setup over all n included)")}
        print(json.dumps(line), flush=True)
    barrier()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
