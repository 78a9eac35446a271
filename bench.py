"""Throughput of the partial wave analysis likelihood hot path on GB300.

One step = one evaluation of NLL(V) and its gradient dNLL/dV* (Eq. 3) over
the whole resident sample: 1M data events x 20 waves, with the normalisation
matrix built once from 5M accepted MC events. Inputs are seeded synthetic
J/psi -> gamma K+ K- shaped samples (no experiment data is available).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line. `value` is device-timed (CUDA events on the launching
stream, L2 flushed between steps); `e2e` times the public host call
(V in from pinned memory, NLL and gradient back) with a wall clock. With
N > 1 (torchrun) every rank runs an independent replica on its own GPU
(weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLL+grad evals/s (1M events, 20 waves, K starts); % HBM / tensor roofline"
UNIT = "evals/s"
N_WAVES, N_DATA, N_MC = 20, 1_000_000, 5_000_000
WORKLOAD = "1M data events x 20 waves (FP32 amplitudes, direct form), M from 5M accepted MC, K=1 per evaluation"
# DRAM bytes (read + write) per launch of the timed kernel from one ncu capture
# (profiles/nll_amp_1M_20waves.md); None once the kernel has changed since.
KERNEL = "nll_amp_kernel<20, 2>"
TRAFFIC_BYTES = 160.145664e6 + 4.291840e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def start_clock_sampler(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def summarise_clocks(path, gpu_index):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
    except FileNotFoundError:
        pass
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_baseline(wl, M, V, budget_s=12.0):
    """The FP64 oracle as it stands (single-threaded C) on the full sample."""
    import oracle
    oracle.nll_amp(wl.A_data, M, V)  # warm (loads the library)
    t0, n = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s or n < 2:
        oracle.nll_amp(wl.A_data, M, V)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full NLL+grad evaluations of the same 1M-event, 20-wave sample "
                      "(M precomputed), FP64 C oracle, 1 thread" % n}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    wl = synth.paper_scale()
    M = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    V = synth.start_points(N_WAVES, 1)[0]
    for _ in range(args.warmup):
        oracle.nll_amp(wl.A_data, M, V)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.nll_amp(wl.A_data, M, V)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_waves": N_WAVES,
                                        "n_data": N_DATA, "n_mc_acc": N_MC},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "each step one full NLL+grad evaluation of the 1M-event sample"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import torch
    import synth
    import paper_1108_5673_gb300 as pwa

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = synth.paper_scale()
    V = synth.start_points(N_WAVES, 1, seed=synth.SEED_STARTS + rank)[0]
    # one explicit stream for the library, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    L = pwa.Likelihood(N_WAVES, device=local, max_k=1, stream=stream.cuda_stream)
    L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    t0 = time.perf_counter()
    M = L.build_norm()
    build_norm_s = time.perf_counter() - t0

    dV = torch.from_numpy(V[None]).cuda()
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    dg = torch.empty(1, N_WAVES, dtype=torch.complex128, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def evict_l2(i):
        # write a buffer larger than L2, then read it back: the sample is evicted
        # and the cache holds clean lines, so no write-back lands in the timed step
        flush.fill_(float(i & 0xff))
        return flush.sum()

    for i in range(args.warmup):
        evict_l2(i)
        L.nll_grad_async(dV, dn, dg)
    assert L.sync() == pwa.PWA_OK

    clock_path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out"))
                              else ".", "bench_clocks_rank%d.csv" % rank)
    sampler = start_clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        evict_l2(i)                      # untimed
        starts[i].record(stream)
        L.nll_grad_async(dV, dn, dg)
        ends[i].record(stream)
    torch.cuda.synchronize()
    status = L.sync()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    # back-to-back (no flush), for reference only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        L.nll_grad_async(dV, dn, dg)
    e1.record(stream)
    torch.cuda.synchronize()
    b2b_ms = e0.elapsed_time(e1) / args.steps
    # end to end through the public host call (V in, NLL + gradient out)
    Vh = V[None].copy()
    for _ in range(3):
        L.nll_grad(Vh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.nll_grad(Vh)
    e2e_s = time.perf_counter() - t0
    if sampler:
        sampler.terminate()
        sampler.wait()

    total_ms_max = total_ms
    e2e_max = e2e_s
    if dist:
        t = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms_max, e2e_max = float(t[0]), float(t[1])
        dist.barrier()
    if rank != 0:
        L.close()
        if dist:
            dist.destroy_process_group()
        return

    value = world * args.steps / (total_ms_max / 1e3)
    e2e_value = world * args.steps / e2e_max
    avg_s = total_ms / args.steps / 1e3
    alg_bytes = 8.0 * N_WAVES * N_DATA
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_s / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_waves": N_WAVES, "n_data": N_DATA, "n_mc_acc": N_MC,
                   "n_mc_gen": wl.n_gen, "K": 1, "form": "amp",
                   "l2": "flushed between timed steps (256 MB write + read back, untimed)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "ms_per_step_back_to_back": b2b_ms, "build_norm_s": build_norm_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES, "peak_kind": peak_kind,
                     "kernel": KERNEL,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * N_WAVES + 8,
                "d2h_bytes_per_step": 8 + 16 * N_WAVES + 8},
        "gpu_launches": args.steps,
        "status": status,
    }
    if sampler:
        out["clocks"] = summarise_clocks(clock_path, local)
    if not args.no_cpu_baseline:
        import oracle
        Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
        out["cpu_baseline"] = cpu_oracle_baseline(wl, Mo, V)
    print(json.dumps(out))
    L.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
