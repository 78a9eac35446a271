"""Throughput of the partial wave analysis likelihood hot path on GB300.

Default workload (`--workload direct`, the headline): one step = one
evaluation of NLL(V) and its gradient dNLL/dV* (Eq. 3) over the whole
resident sample, 1M data events x 20 waves, direct amplitude form, with the
normalisation matrix built once from 5M accepted MC events. Inputs are seeded
synthetic J/psi -> gamma K+ K- shaped samples (no experiment data exists here).

Other workloads (one JSON line each, same keys):
  table   the same sample and evaluation in the per-event table form (Sec. 2)
  tc      K = 256 starting parameter sets at once on the tensor cores:
          4M events x 32 waves, M from 10M accepted MC (--precision bfp16|bfp8)
  res     free masses and widths of 4 of 20 Breit-Wigner waves: 2M data events,
          5M accepted MC, amplitudes recomputed every call
  models  64 trial models (n_waves 8..48, 100k..2M data events, MC 2x data),
          K = 16 parameter sets each, one graph launch per step
  hessian the FUMILI Hessian (2N x 2N over Re V, Im V) of the direct-form
          sample (1M events x 20 waves); one step = one Hessian
  weights projection weights I / N_gen of the 5M accepted MC events of the
          same sample into a device buffer; one step = one pass
  incoh   incoherent sum over 2 unobserved components per event (I = sum_l
          |sum_a V_a A_a^l|^2): 1M data events x 20 waves x 2, direct form
  incoh_table  the same sample in the table form (table bytes independent of
          the number of components)
  ampgen  amplitudes BW x Y_l^m of 5M events x 20 waves generated on the
          device from their kinematics (FP64, rounded to complex64)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload direct|table|tc|res|models|hessian|weights|incoh|incoh_table|ampgen]

`value` is device-timed (CUDA events on the launching stream; L2 flushed
between steps where the inputs fit in it); `e2e` times the public host call
(inputs from host memory, results back) with a wall clock. With N > 1
(torchrun) every rank runs an independent replica on its own GPU (weak
scaling, no collective on the data path); rank 0 prints.

The default line also carries, timed in the same run on the same GPU with
fewer steps, `secondary`: the table form of the headline sample and K = 256
sets on the tensor cores (4M events x 32 waves, generated on the device),
each with its own roofline and clocks (--no-secondary skips them); and next
to `cpu_baseline` (the oracle on one thread) `cpu_baseline_all_cores` (the
unchanged oracle on one chunk of events per host core, spawned processes).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLL+grad evals/s (1M events, 20 waves, K starts); % HBM / tensor roofline"
UNIT = "evals/s"
N_WAVES, N_DATA, N_MC = 20, 1_000_000, 5_000_000
WORKLOAD = "1M data events x 20 waves (FP32 amplitudes, direct form), M from 5M accepted MC, K=1 per evaluation"
# DRAM bytes (read + write) per step of the timed kernel from one ncu
# capture of the current kernel, or None where there is none.
TRAFFIC = {"direct": 160.139776e6 + 3.347968e6,
           "table": 1600.119e6 + 3.221760e6,
           "tc": 2 * (1024.872e6 + 3.708160e6),        # a step is two launches of 128 sets
           "res": 1148.176e6 + 3.313920e6,
           "models": None,
           "hessian": 160.091648e6 + 3.346944e6,
           "weights": 800.125184e6 + 21.052672e6,
           "incoh": 320.158464e6 + 3.042048e6,
           "incoh_table": None,   # the table kernel's capture is of the coherent sample
           "ampgen": 278.9e6 + 962.9e6,   # FP64-bound; DRAM bytes for reference
           "direct_4M_32": None,   # kernel changed since its capture (four-warp groups, amplitudes re-read)
           "cov_ampgen": 1233.902e6 + 2723.644e6}   # FP64-bound; DRAM bytes for reference
KERNELS = {"direct": "nll_amp_kernel<20, 2>", "table": "nll_table_kernel<20>",
           "tc": "batched_kernel<64, 2>", "res": "nll_res_tma_kernel<20, 4>",
           "models": "batched_items_kernel<2> (all models, one launch)", "hessian": "hess_tc_kernel<20>",
           "weights": "nll_amp_kernel<20, 2, 1, true> (weights mode)", "incoh": "nll_amp_kernel<20, 2, 2>",
           "incoh_table": "nll_table_kernel<20>", "ampgen": "amp_gen_kernel",
           "direct_4M_32": "nll_amp_kernel<32, 2>", "cov_ampgen": "cov_amp_kernel"}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64 (nominal)
HBM_NOMINAL_GBS = 7900.0     # GB300 HBM3e (nominal), beside the measured copy peak
BF16_NOMINAL_TFLOPS = 2250.0  # GB300 dense bf16 (nominal)
DEFAULT_STEPS = {"direct": 3000, "table": 1000, "tc": 300, "res": 1000, "models": 100,
                 "hessian": 2000, "weights": 2000, "incoh": 1500, "incoh_table": 1000,
                 "ampgen": 100, "direct_4M_32": 500, "cov_ampgen": 100}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm": p["hbm_gbs"], "bf16": p["bf16_tflops"],
                "bf16_sustained": p["bf16_tflops_sustained"], "kind": "measured"}
    except Exception:
        return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "kind": "fallback"}


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


def timed_oracle(fn, budget_s):
    """Calls fn() until budget_s has passed (at least twice); seconds per call."""
    fn()
    t0, n = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s or n < 2:
        fn()
        n += 1
    return (time.perf_counter() - t0) / n, n


_CHUNK = {}


def _oracle_chunk_init(shm_name, shape, M, V):
    from multiprocessing import shared_memory
    _CHUNK["shm"] = shared_memory.SharedMemory(name=shm_name)
    _CHUNK["A"] = np.ndarray(shape, dtype=np.complex128, buffer=_CHUNK["shm"].buf)
    _CHUNK["M"], _CHUNK["V"] = M, V


def _oracle_chunk_eval(bounds):
    import oracle
    lo, hi = bounds
    return oracle.nll_amp(_CHUNK["A"][lo:hi], _CHUNK["M"], _CHUNK["V"])[0]


def oracle_all_cores(A, M, V, budget_s):
    """The oracle as it stands on all host cores: the events split into one
    contiguous chunk per core, each evaluated by oracle.nll_amp in its own
    spawned process (the MC term is added per chunk; its cost is O(N^2)).
    Returns (seconds per full evaluation, steps timed, processes)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    P = os.cpu_count() or 1
    A = np.ascontiguousarray(A, dtype=np.complex128)
    shm = shared_memory.SharedMemory(create=True, size=A.nbytes)
    try:
        np.ndarray(A.shape, dtype=np.complex128, buffer=shm.buf)[:] = A
        n = A.shape[0]
        bounds = [(n * k // P, n * (k + 1) // P) for k in range(P)]
        with mp.get_context("spawn").Pool(P, initializer=_oracle_chunk_init,
                                          initargs=(shm.name, A.shape, M, V)) as pool:
            pool.map(_oracle_chunk_eval, bounds)          # warm-up (imports, library load)
            t0, k = time.perf_counter(), 0
            while time.perf_counter() - t0 < budget_s or k < 2:
                pool.map(_oracle_chunk_eval, bounds)
                k += 1
            dt = (time.perf_counter() - t0) / k
    finally:
        shm.close()
        shm.unlink()
    return dt, k, P


# ---- workloads: each sets up the library and returns a Job ---------------------

class Job:
    """step(): enqueue one step on `stream` (device-resident inputs);
    host_step(): one public host call (inputs from host memory, results back);
    outputs(): optional, the last step's results as a numpy array (the line
    reports whether they are all finite)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def outputs_finite(job):
    """Whether the last step's results are all finite (None: not checked)."""
    f = getattr(job, "outputs", None)
    if f is None:
        return None
    return bool(np.all(np.isfinite(np.asarray(f()))))


def job_direct(pwa, torch, stream, local, rank, form="amp"):
    import synth
    wl = synth.paper_scale()
    V = synth.start_points(N_WAVES, 1, seed=synth.SEED_STARTS + rank)[0]
    forms = pwa.PWA_FORM_AMP | (pwa.PWA_FORM_TABLE if form == "table" else 0)
    L = pwa.Likelihood(N_WAVES, device=local, forms=forms, max_k=1, stream=stream.cuda_stream)
    L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    t0 = time.perf_counter()
    L.build_norm()
    build_norm_s = time.perf_counter() - t0
    if form == "table":
        L.set_form(pwa.PWA_FORM_TABLE)
    dV = torch.from_numpy(V[None]).cuda()
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    dg = torch.empty(1, N_WAVES, dtype=torch.complex128, device="cuda")
    Vh = V[None].copy()

    def cpu_baseline():
        import oracle
        Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
        if form == "table":
            n = 100_000
            T = oracle.table(wl.A_data[:n])
            dt, k = timed_oracle(lambda: oracle.nll_table(T, Mo, V), 12.0)
            return {"value": 1.0 / (dt * N_DATA / n), "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": "%d table-form NLL+grad evaluations of the first 100k events (FP64 C "
                              "oracle, 1 thread), scaled to the 1M-event sample" % k}
        dt, k = timed_oracle(lambda: oracle.nll_amp(wl.A_data, Mo, V), 12.0)
        return {"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d full NLL+grad evaluations of the same 1M-event, 20-wave sample "
                          "(M precomputed), FP64 C oracle, 1 thread" % k}

    def cpu_baseline_all():
        import oracle
        Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
        dt, k, P = oracle_all_cores(wl.A_data, Mo, V, 8.0)
        return {"value": 1.0 / dt, "unit": UNIT, "cores": P, "kind": "oracle",
                "sample": "%d full NLL+grad evaluations of the same sample, the 1M events split "
                          "into %d chunks evaluated by the unchanged FP64 C oracle in %d spawned "
                          "processes" % (k, P, P)}

    table = form == "table"
    return Job(
        name=form if table else "direct", lib=L,
        step=lambda: L.nll_grad_async(dV, dn, dg), host_step=lambda: L.nll_grad(Vh),
        outputs=lambda: np.concatenate([dn.cpu().numpy(), dg.cpu().numpy().view(np.float64).ravel()]),
        sync=L.sync, evals_per_step=1, launches_per_step=1, flush=True,
        workload=("1M data events x 20 waves (FP32 per-event table of 400 floats, table form), "
                  "M from 5M accepted MC, K=1 per evaluation") if table else WORKLOAD,
        config={"n_waves": N_WAVES, "n_data": N_DATA, "n_mc_acc": N_MC, "n_mc_gen": wl.n_gen,
                "K": 1, "form": form, "build_norm_s": build_norm_s},
        roof={"bound": "hbm", "bytes": (4.0 * N_WAVES ** 2 if table else 8.0 * N_WAVES) * N_DATA},
        dtype="f32", h2d=16 * N_WAVES + 8, d2h=8 + 16 * N_WAVES + 8, cpu_baseline=cpu_baseline,
        cpu_baseline_all=None if table else cpu_baseline_all)


def job_tc(pwa, torch, stream, local, rank, precision="bfp16", gen="numpy"):
    import synth
    N, n, n_mc, K = 32, 4_000_000, 10_000_000, 256
    if gen == "torch":
        # the same sample shape from the torch generator on the device (the
        # host generator takes ~40 s for these 14M events)
        A_d, A_m, n_gen = synth.torch_mixture_workload(synth.waves_linear(N), n, n_mc,
                                                       synth.SEED_DATA + rank)
        wl = synth.Workload("pwa_4M_events_32_waves", synth.waves_linear(N), A_d, A_m, n_gen,
                            synth.random_V(N, synth.SEED_DATA + rank))
    else:
        wl = synth.multistart_scale()
    Vs = synth.start_points(N, K, seed=synth.SEED_STARTS + rank) * 2.0
    prec = pwa.PWA_PREC_BFP8 if precision == "bfp8" else pwa.PWA_PREC_BFP16
    L = pwa.Likelihood(N, device=local, forms=pwa.PWA_FORM_TC, max_k=K, stream=stream.cuda_stream,
                       precision=prec)
    L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    t0 = time.perf_counter()
    L.build_norm()
    build_norm_s = time.perf_counter() - t0
    L.set_form(pwa.PWA_FORM_TC)
    dV = torch.from_numpy(Vs).cuda()
    dn = torch.empty(K, dtype=torch.float64, device="cuda")
    dg = torch.empty(K, N, dtype=torch.complex128, device="cuda")

    def cpu_baseline():
        import oracle
        sub = 200_000
        A = wl.A_data[:sub]
        Mo = oracle.norm_matrix_blas(wl.A_mc[:1_000_000], wl.n_gen)
        dt, k = timed_oracle(lambda: oracle.nll_amp(A, Mo, Vs[0]), 12.0)
        return {"value": 1.0 / (dt * n / sub), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d NLL+grad evaluations of one parameter set on the first 200k of the "
                          "4M events (FP64 C oracle, 1 thread), scaled to one evaluation of the "
                          "full sample" % k}

    return Job(
        name="tc", lib=L, step=lambda: L.nll_grad_async(dV, dn, dg), host_step=lambda: L.nll_grad(Vs),
        outputs=lambda: np.concatenate([dn.cpu().numpy(), dg.cpu().numpy().view(np.float64).ravel()]),
        sync=L.sync, evals_per_step=K, launches_per_step=2 * 3, flush=False,
        workload="4M data events x 32 waves, K=256 parameter sets per call on the tensor cores "
                 "(%s amplitudes, 24-bit V slices), M from 10M accepted MC" % precision,
        config={"n_waves": N, "n_data": n, "n_mc_acc": n_mc, "n_mc_gen": wl.n_gen, "K": K,
                "form": "tc", "precision": precision, "build_norm_s": build_norm_s},
        roof={"bound": "tensor", "flops": 16.0 * N * K * n},
        dtype="bf16", h2d=16 * N * K, d2h=8 * K + 16 * N * K, cpu_baseline=cpu_baseline)


def job_direct32(pwa, torch, stream, local, rank):
    """The plain single-fit form (direct, FP32 amplitudes, one parameter set
    per call) on the tensor-core form's sample, 4M events x 32 waves: the
    denominator of the batched form's speed-up on the same GPU."""
    import synth
    N, n, n_mc = 32, 4_000_000, 10_000_000
    A_d, A_m, n_gen = synth.torch_mixture_workload(synth.waves_linear(N), n, n_mc,
                                                   synth.SEED_DATA + rank)
    V = synth.start_points(N, 1, seed=synth.SEED_STARTS + rank)[0] * 2.0
    L = pwa.Likelihood(N, device=local, forms=pwa.PWA_FORM_AMP, max_k=1, stream=stream.cuda_stream)
    L.load_events(A_d, A_m, n_gen)
    del A_m
    L.build_norm()
    dV = torch.from_numpy(V[None]).cuda()
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    dg = torch.empty(1, N, dtype=torch.complex128, device="cuda")
    Vh = V[None].copy()

    def cpu_baseline():
        import oracle
        sub = 200_000
        A = A_d[:sub].cpu().numpy()
        Mo = L.M if L.M is not None else L.build_norm()
        dt, k = timed_oracle(lambda: oracle.nll_amp(A, Mo, V), 12.0)
        return {"value": 1.0 / (dt * n / sub), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d NLL+grad evaluations on the first 200k of the 4M events (FP64 C "
                          "oracle, 1 thread, M as built on the GPU), scaled to the full sample" % k}

    return Job(
        name="direct_4M_32", lib=L, step=lambda: L.nll_grad_async(dV, dn, dg),
        outputs=lambda: np.concatenate([dn.cpu().numpy(), dg.cpu().numpy().view(np.float64).ravel()]),
        host_step=lambda: L.nll_grad(Vh), sync=L.sync, evals_per_step=1, launches_per_step=1,
        flush=False,
        workload="4M data events x 32 waves (FP32 amplitudes, direct form), M from 10M accepted "
                 "MC, K=1 per evaluation (the tensor-core form's sample)",
        config={"n_waves": N, "n_data": n, "n_mc_acc": n_mc, "n_mc_gen": n_gen, "K": 1,
                "form": "amp"},
        roof={"bound": "hbm", "bytes": 8.0 * N * n},
        dtype="f32", h2d=16 * N + 8, d2h=8 + 16 * N + 8, cpu_baseline=cpu_baseline)


def job_res(pwa, torch, stream, local, rank):
    import synth
    N, R, n, n_mc = 20, 4, 2_000_000, 5_000_000
    wl = synth.free_resonance_scale()
    V = synth.start_points(N, 1, seed=synth.SEED_STARTS + rank)[0]
    mass, width = wl.mass * 1.01, wl.width * 0.95
    L = pwa.Likelihood(N, device=local, max_k=1, stream=stream.cuda_stream)
    L.load_resonance_events(wl)

    def cpu_baseline():
        import oracle
        sd, sm = 100_000, 250_000
        args = (wl.m_data[:sd].astype(np.float64), wl.Y_data[:sd], wl.Afix_data[:sd],
                wl.m_mc[:sm].astype(np.float64), wl.Y_mc[:sm], wl.Afix_mc[:sm], float(wl.n_gen))
        dt, k = timed_oracle(lambda: oracle.nll_res(*args, V, mass, width), 12.0)
        return {"value": 1.0 / (dt * (n + n_mc) / (sd + sm)), "unit": UNIT, "cores": 1,
                "kind": "oracle",
                "sample": "%d free-resonance NLL+gradient evaluations on the first 100k data and "
                          "250k MC events (FP64 C oracle, 1 thread), scaled to the full 2M + 5M "
                          "events" % k}

    import torch as _t
    dV = _t.from_numpy(np.ascontiguousarray(V)).cuda()
    dm = _t.tensor(mass, dtype=_t.float64, device="cuda")
    dw = _t.tensor(width, dtype=_t.float64, device="cuda")
    dout = _t.empty(1 + 2 * N + 2 * R, dtype=_t.float64, device="cuda")
    return Job(
        name="res", lib=L, step=lambda: L.nll_grad_res_async(dV, dm, dw, dout),
        host_step=lambda: L.nll_grad_res(V, mass, width), sync=L.sync,
        evals_per_step=1, launches_per_step=1, flush=False,
        workload="free masses and widths of 4 of 20 Breit-Wigner waves: 2M data + 5M accepted MC "
                 "events (m, Y of the free waves, fixed amplitudes; FP32), BW recomputed per call",
        config={"n_waves": N, "n_free": R, "n_data": n, "n_mc_acc": n_mc, "n_mc_gen": wl.n_gen,
                "K": 1, "form": "res"},
        roof={"bound": "hbm", "bytes": 4.0 * (1 + 2 * N) * (n + n_mc)},
        dtype="f32", h2d=16 * N + 16 * R + 8, d2h=8 + 16 * N + 16 * R, cpu_baseline=cpu_baseline)


def job_models(pwa, torch, stream, local, rank):
    import synth
    spec = synth.model_batch_spec()
    K = 16
    B = pwa.ModelBatch([s[0] for s in spec], K, device=local, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    for j, (nw, nd, seed) in enumerate(spec):
        A_d, A_m, n_gen = synth.torch_mixture_workload(synth.waves_linear(nw), nd, 2 * nd, seed + rank)
        B.load_model(j, A_d, A_m, n_gen)
        del A_d, A_m
    torch.cuda.empty_cache()
    load_s = time.perf_counter() - t0
    Vs = [synth.start_points(s[0], K, seed=s[2] + 7) * 2.0 for s in spec]

    def cpu_baseline():
        import oracle
        nw, nd, seed = spec[0]
        A_d, A_m, n_gen = synth.torch_mixture_workload(synth.waves_linear(nw), 50_000, 100_000, seed)
        A_d, A_m = A_d.cpu().numpy(), A_m.cpu().numpy()
        Mo = oracle.norm_matrix(A_m, n_gen)
        dt, k = timed_oracle(lambda: oracle.nll_amp(A_d, Mo, Vs[0][0]), 10.0)
        per_wave_event = dt / (50_000 * nw)
        t_call = sum(K * s[0] * s[1] for s in spec) * per_wave_event
        return {"value": 64 * K / t_call, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d NLL+grad evaluations of model 0 (%d waves) on 50k events (FP64 C "
                          "oracle, 1 thread), scaled by waves x events to 16 sets of each of the "
                          "64 models" % (k, nw)}

    last = {}

    def step():
        last["r"] = B.nll_grad(Vs)

    return Job(
        name="models", lib=B, step=step, host_step=lambda: B.nll_grad(Vs),
        outputs=lambda: np.concatenate([np.ravel(x) for x in last["r"][0]] +
                                       [np.ravel(x).view(np.float64) for x in last["r"][1]]),
        sync=lambda: B.last_status, evals_per_step=64 * K, launches_per_step=3,
        flush=False,
        workload="64 trial models (n_waves 8..48, 100k..2M data events each, MC 2x data, 63.4M "
                 "data events in all), K=16 parameter sets per model, one persistent launch over "
                 "(model, tile range) work items",
        config={"n_models": 64, "K": K, "n_data_total": sum(s[1] for s in spec),
                "n_waves_mean": float(np.mean([s[0] for s in spec])), "form": "tc",
                "precision": "bfp16", "load_and_norm_s": load_s},
        # K = 16 sets: 16 N K flops over 8 N bytes per event = 2K = 32 flop/B, a tenth of
        # the machine balance (bf16 peak / HBM), so the step is bound by reading the
        # amplitudes once per model: 8 N_m bytes per event of model m
        roof={"bound": "hbm", "bytes": float(sum(8.0 * s[0] * s[1] for s in spec)),
              "flops": float(sum(16.0 * s[0] * K * s[1] for s in spec))},
        dtype="bf16", h2d=16 * K * sum(s[0] for s in spec),
        d2h=8 * 64 * K + 16 * K * sum(s[0] for s in spec), cpu_baseline=cpu_baseline,
        note="value and e2e both time the host call (V of all models in, results out, ~0.5 MB "
             "each way)")


def job_incoh(pwa, torch, stream, local, rank, form="amp"):
    """Incoherent sum over 2 components: 1M data events x 20 waves x 2, M
    from 2M accepted MC events x 2 components."""
    import synth
    L_, n_mc = 2, 2_000_000
    wl = synth.incoherent_workload("incoh_1M_events_20_waves_2_components",
                                   synth.waves_linear(N_WAVES), N_DATA, n_mc, n_lambda=L_)
    V = synth.start_points(N_WAVES, 1, seed=synth.SEED_STARTS + rank)[0]
    table = form == "table"
    forms = pwa.PWA_FORM_TABLE if table else pwa.PWA_FORM_AMP
    L = pwa.Likelihood(N_WAVES, device=local, forms=forms, max_k=1, stream=stream.cuda_stream)
    L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    t0 = time.perf_counter()
    L.build_norm()
    build_norm_s = time.perf_counter() - t0
    dV = torch.from_numpy(V[None]).cuda()
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    dg = torch.empty(1, N_WAVES, dtype=torch.complex128, device="cuda")
    Vh = V[None].copy()

    def cpu_baseline():
        import oracle
        sub = 200_000
        Mo = oracle.norm_matrix_incoh(wl.A_mc[:200_000], wl.n_gen)
        dt, k = timed_oracle(lambda: oracle.nll_incoh(wl.A_data[:sub], Mo, V), 10.0)
        return {"value": 1.0 / (dt * N_DATA / sub), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d incoherent NLL+grad evaluations of the first 200k events (FP64 C "
                          "oracle, 1 thread), scaled to the 1M-event sample" % k}

    return Job(
        name="incoh_table" if table else "incoh", lib=L,
        step=lambda: L.nll_grad_async(dV, dn, dg), host_step=lambda: L.nll_grad(Vh),
        sync=L.sync, evals_per_step=1, launches_per_step=1, flush=False,
        metric="NLL+grad evals/s, incoherent sum over 2 components (1M events, 20 waves); "
               "% HBM roofline",
        workload="1M data events x 20 waves x 2 incoherent components (FP32 amplitudes, %s), "
                 "M from 2M accepted MC x 2 components, K=1 per evaluation"
                 % ("per-event table of 400 floats, table form" if table else "direct form"),
        config={"n_waves": N_WAVES, "n_lambda": L_, "n_data": N_DATA, "n_mc_acc": n_mc,
                "n_mc_gen": wl.n_gen, "K": 1, "form": form, "build_norm_s": build_norm_s},
        roof={"bound": "hbm", "bytes": (4.0 * N_WAVES ** 2 if table else 8.0 * L_ * N_WAVES) * N_DATA},
        dtype="f32", h2d=16 * N_WAVES + 8, d2h=8 + 16 * N_WAVES + 8, cpu_baseline=cpu_baseline)


def ampgen_flops(waves):
    """FP64 operations per event of the generator as written: 6 per power of
    e^{i phi} up to max |m|, and per wave 4 per step of P_m^m, 7 per step of
    the recurrence in l, 20 for the normalisation, Breit-Wigner and complex
    product (divisions and the one sincos counted as one operation each)."""
    mx = max(abs(w.m) for w in waves)
    return 6 * mx + 1 + sum(4 * abs(w.m) + 7 * max(0, w.l - abs(w.m) - 1) + 20 for w in waves)


def job_ampgen(pwa, torch, stream, local, rank):
    import synth
    n = N_MC
    waves = synth.waves_linear(N_WAVES)
    ev, _ = synth.mc_sample(n, seed=synth.SEED_MC + rank)
    kin_h = np.stack([ev["m"], ev["costh"], ev["phi"]], axis=1)
    kin = torch.from_numpy(kin_h).cuda()
    out = torch.empty(n, N_WAVES, dtype=torch.complex64, device="cuda")
    L = pwa.Likelihood(N_WAVES, device=local, max_k=1, stream=stream.cuda_stream)

    def cpu_baseline():
        import oracle
        sub = 200_000
        dt, k = timed_oracle(lambda: oracle.amplitudes(ev["m"][:sub], ev["costh"][:sub],
                                                       ev["phi"][:sub], waves), 10.0)
        return {"value": 1.0 / (dt * n / sub), "unit": "passes/s", "cores": 1, "kind": "oracle",
                "sample": "%d amplitude evaluations of the first 200k events x 20 waves (FP64 C "
                          "oracle, 1 thread), scaled to 5M events" % k}

    return Job(
        name="ampgen", lib=L, step=lambda: L.amplitudes(waves, kin, out),
        host_step=lambda: L.amplitudes(waves, kin_h), sync=lambda: L.last_status,
        evals_per_step=1, launches_per_step=1, flush=False,
        metric="amplitude-generation passes/s (5M events x 20 waves, BW x Y_l^m); % FP64 peak",
        unit="passes/s",
        workload="amplitudes BW x Y_l^m of 5M events x 20 waves from device-resident "
                 "kinematics (FP64 arithmetic, complex64 out to a device buffer)",
        config={"n_waves": N_WAVES, "n_events": n, "flops_per_event": ampgen_flops(waves)},
        roof={"bound": "alu", "flops": float(ampgen_flops(waves)) * n},
        dtype="f64", h2d=24 * n, d2h=8 * N_WAVES * n, cpu_baseline=cpu_baseline,
        note="e2e passes host kinematics in (120 MB) and takes the amplitudes back (800 MB)")


def cov_ampgen_flops(n_waves):
    """FP64 operations per event of the covariant generator as written, each
    +, -, x, fma, division and square root counted as one: ~357 for the
    four-vectors, r~, the barrier factor, the photon polarisations and the
    spin-0 and spin-2 contractions of the four components (every metric dot
    product counted in full, 7 operations), and ~33 per wave for the
    Breit-Wigner and the four complex products."""
    return 357 + 33 * n_waves


def job_cov_ampgen(pwa, torch, stream, local, rank):
    import synth
    n, N = N_MC, 12
    waves = synth.cov_waves(N)
    p3_h, _ = synth.radiative_events(n, np.random.default_rng(synth.SEED_MC + rank))
    p3 = torch.from_numpy(p3_h).cuda()
    out = torch.empty(n, 4, N, dtype=torch.complex64, device="cuda")
    L = pwa.Likelihood(N, device=local, max_k=1, stream=stream.cuda_stream)

    def cpu_baseline():
        import oracle
        sub = 200_000
        dt, k = timed_oracle(lambda: oracle.covariant_amplitudes(p3_h[:sub], waves), 10.0)
        return {"value": 1.0 / (dt * n / sub), "unit": "passes/s", "cores": 1, "kind": "oracle",
                "sample": "%d covariant amplitude evaluations of the first 200k events x 12 waves "
                          "x 4 components (FP64 C oracle, 1 thread), scaled to 5M events" % k}

    return Job(
        name="cov_ampgen", lib=L, step=lambda: L.covariant_amplitudes(waves, p3, out),
        host_step=lambda: L.covariant_amplitudes(waves, p3_h), sync=lambda: L.last_status,
        evals_per_step=1, launches_per_step=1, flush=False,
        metric="covariant amplitude passes/s (5M J/psi -> gamma K+ K- events x 12 waves x 4 "
               "components); % FP64 peak",
        unit="passes/s",
        workload="covariant tensor amplitudes of J/psi -> gamma X, X -> K+ K- (spins 0 and 2) for "
                 "5M events x 12 waves x 4 components from device-resident 3-momenta (FP64 "
                 "arithmetic, complex64 out to a device buffer)",
        config={"n_waves": N, "n_events": n, "components": 4,
                "flops_per_event": cov_ampgen_flops(N)},
        roof={"bound": "alu", "flops": float(cov_ampgen_flops(N)) * n},
        dtype="f64", h2d=72 * n, d2h=32 * N * n, cpu_baseline=cpu_baseline,
        note="e2e passes host 3-momenta in (360 MB) and takes the amplitudes back (1.9 GB)")


def job_fit_extra(pwa, torch, stream, local, rank, what):
    """FUMILI Hessian of the 1M-event sample, or the projection weights of its
    5M accepted MC events (host V in; H to the host, or w into a device buffer)."""
    import synth
    wl = synth.paper_scale()
    V = synth.start_points(N_WAVES, 1, seed=synth.SEED_STARTS + rank)[0]
    L = pwa.Likelihood(N_WAVES, device=local, max_k=1, stream=stream.cuda_stream)
    L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    L.build_norm()
    if what == "hessian":
        def cpu_baseline():
            import oracle
            sub = 20_000
            dt, k = timed_oracle(lambda: oracle.hessian(wl.A_data[:sub], V), 10.0)
            return {"value": 1.0 / (dt * N_DATA / sub), "unit": "Hessians/s", "cores": 1,
                    "kind": "oracle",
                    "sample": "%d FUMILI Hessians of the first 20k events (FP64 C oracle, "
                              "1 thread), scaled to the 1M-event sample" % k}

        P = 2 * N_WAVES
        dV = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        dH = torch.empty(P, P, dtype=torch.float64, device="cuda")
        return Job(
            name="hessian", lib=L, step=lambda: L.hessian_async(dV, dH),
            host_step=lambda: L.hessian(V), sync=L.sync,
            evals_per_step=1, launches_per_step=2, flush=True,
            metric="FUMILI Hessian evals/s (1M events, 20 waves); % HBM roofline",
            unit="Hessians/s",
            workload="FUMILI Hessian (40 x 40 over Re V, Im V) of 1M data events x 20 waves "
                     "(FP32 amplitudes), M from 5M accepted MC",
            config={"n_waves": N_WAVES, "n_data": N_DATA, "n_mc_acc": N_MC, "K": 1},
            roof={"bound": "hbm", "bytes": 8.0 * N_WAVES * N_DATA},
            dtype="f32", h2d=16 * N_WAVES, d2h=8 * P * P + 4, cpu_baseline=cpu_baseline)

    out = torch.empty(N_MC, dtype=torch.float32, device="cuda")

    def cpu_baseline():
        import oracle
        sub = 500_000
        dt, k = timed_oracle(lambda: oracle.mc_weights(wl.A_mc[:sub], V, wl.n_gen), 10.0)
        return {"value": 1.0 / (dt * N_MC / sub), "unit": "passes/s", "cores": 1, "kind": "oracle",
                "sample": "%d weight passes over the first 500k accepted MC events (FP64 C oracle, "
                          "1 thread), scaled to the 5M events" % k}

    step = lambda: L.mc_weights(V, out)
    return Job(
        name="weights", lib=L, step=step, host_step=lambda: L.mc_weights(V),
        sync=lambda: L.last_status, evals_per_step=1, launches_per_step=1, flush=False,
        metric="projection-weight passes/s (5M accepted MC events, 20 waves); % HBM roofline",
        unit="passes/s",
        workload="projection weights I(Omega_j) / N_gen of 5M accepted MC events x 20 waves (FP32 "
                 "amplitudes, FP32 weights into a device buffer)",
        config={"n_waves": N_WAVES, "n_mc_acc": N_MC, "n_mc_gen": wl.n_gen},
        roof={"bound": "hbm", "bytes": (8.0 * N_WAVES + 4.0) * N_MC},
        dtype="f32", h2d=16 * N_WAVES, d2h=4 * N_MC, cpu_baseline=cpu_baseline,
        note="value times the call writing into a device buffer; e2e the call returning the "
             "weights to host memory (20 MB)")


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
                                        "n_data": N_DATA, "n_mc_acc": N_MC, "n_mc_gen": wl.n_gen,
                                        "K": 1, "form": "amp"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "each step one full NLL+grad evaluation of the 1M-event sample"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def max_over_ranks(dist, values, device):
    """The per-rank timings [device ms, end-to-end s] reduced to their maximum
    over ranks (the slowest replica sets the job's time), followed by a
    barrier; values unchanged without a process group."""
    if not dist:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return [float(x) for x in t]


def job_value(world, evals_per_step, steps, total_ms_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs its own replica)."""
    return world * evals_per_step * steps / (total_ms_max / 1e3)


def matmul_peaks(reps=50, n=8192):
    """Library GEMM rates on this GPU, for the roofline of a TF32 operand
    choice: torch.matmul n^3 in TF32, BF16 and plain FP32, each timed with
    CUDA events over `reps` back-to-back products after 5 warm-ups (2 n^3
    flops each), with the SM clocks sampled meanwhile. Prints one JSON line."""
    import torch
    dev = torch.device("cuda", 0)
    clock_path = os.path.join(tempfile.gettempdir(), "matmul_peaks_clocks.csv")
    sampler = start_clock_sampler(clock_path)
    out = {}
    for name, dt, tf32 in (("tf32", torch.float32, True), ("bf16", torch.bfloat16, False),
                           ("fp32", torch.float32, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        c = torch.empty(n, n, device=dev, dtype=dt)
        for _ in range(5):
            torch.matmul(a, b, out=c)
        r = reps if name != "fp32" else max(reps // 5, 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(r):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / r
        out[name] = {"ms_per_product": ms, "tflops": 2.0 * n ** 3 / ms / 1e9, "products": r}
        del a, b, c
        torch.cuda.empty_cache()
    clocks = None
    if sampler:
        sampler.terminate()
        sampler.wait()
        clocks = summarise_clocks(clock_path, 0)
    out["tf32_over_bf16"] = out["tf32"]["tflops"] / out["bf16"]["tflops"]
    print(json.dumps({"matmul_peaks": out, "n": n, "clocks": clocks,
                      "gpu": torch.cuda.get_device_name(0)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="direct", choices=["direct", "table", "tc", "res", "models", "hessian", "weights",
                             "incoh", "incoh_table", "ampgen", "direct_4M_32", "cov_ampgen"])
    ap.add_argument("--precision", default="bfp16", choices=["bfp16", "bfp8"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the table and tensor-core forms in the default line")
    ap.add_argument("--tune", action="store_true",
                    help="run the library's autotuner on the loaded sample (no cache) before "
                         "timing; its choice is reported in config.autotune")
    ap.add_argument("--matmul-peaks", action="store_true",
                    help="time library GEMMs (TF32, BF16, FP32 8192^3) and print their rates")
    args = ap.parse_args()
    if args.matmul_peaks:
        return matmul_peaks()
    if args.steps is None:
        args.steps = DEFAULT_STEPS[args.workload] if args.impl == "gb300" else 3
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import torch
    import paper_1108_5673_gb300 as pwa

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # one explicit stream for the library, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.workload in ("direct", "table"):
        job = job_direct(pwa, torch, stream, local, rank, form="table" if args.workload == "table" else "amp")
    elif args.workload == "tc":
        job = job_tc(pwa, torch, stream, local, rank, args.precision)
    elif args.workload == "res":
        job = job_res(pwa, torch, stream, local, rank)
    elif args.workload == "direct_4M_32":
        job = job_direct32(pwa, torch, stream, local, rank)
    elif args.workload == "ampgen":
        job = job_ampgen(pwa, torch, stream, local, rank)
    elif args.workload == "cov_ampgen":
        job = job_cov_ampgen(pwa, torch, stream, local, rank)
    elif args.workload in ("incoh", "incoh_table"):
        job = job_incoh(pwa, torch, stream, local, rank, "table" if args.workload == "incoh_table" else "amp")
    elif args.workload in ("hessian", "weights"):
        job = job_fit_extra(pwa, torch, stream, local, rank, args.workload)
    else:
        job = job_models(pwa, torch, stream, local, rank)

    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def evict_l2(i):
        # write a buffer larger than L2, then read it back: the sample is evicted
        # and the cache holds clean lines, so no write-back lands in the timed step
        flush.fill_(float(i & 0xff))
        return flush.sum()

    peaks = measured_peaks()
    tuned = None
    if args.tune and hasattr(job.lib, "autotune"):
        tuned = job.lib.autotune(None)
    m = measure(job, args.steps, args.warmup, evict_l2, stream, dist, rank, local, pwa, torch)
    total_ms_max, e2e_max = max_over_ranks(dist, [m["total_ms"], m["e2e_s"]], "cuda")
    if rank != 0:
        job.lib.close()
        if dist:
            dist.destroy_process_group()
        return

    ev = job.evals_per_step
    value = job_value(world, ev, args.steps, total_ms_max)
    e2e_value = world * ev * args.steps / e2e_max
    config = {"workload": job.workload}
    config.update(job.config)
    config.update({"l2": "flushed between timed steps (256 MB write + read back, untimed)"
                   if job.flush else "inputs larger than L2 (129 MB), no flush",
                   "parallelism": "replicas" if world > 1 else "single",
                   "ms_per_step_back_to_back": m["b2b_ms"]})
    if getattr(job, "note", None):
        config["note"] = job.note
    if tuned is not None:
        config["autotune"] = tuned
    out = {
        "metric": getattr(job, "metric", METRIC), "value": value,
        "unit": getattr(job, "unit", UNIT), "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": job.dtype, "data": "synthetic",
        "config": config, "roofline": roofline(job, m["total_ms"] / args.steps / 1e3, peaks),
        "e2e": {"value": e2e_value, "unit": getattr(job, "unit", UNIT), "h2d_bytes_per_step": job.h2d,
                "d2h_bytes_per_step": job.d2h},
        "gpu_launches": job.launches_per_step * args.steps,
        "status": m["status"],
        "outputs_finite": m["finite"],
    }
    if m["clocks"] is not None:
        out["clocks"] = m["clocks"]
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = job.cpu_baseline()
        if getattr(job, "cpu_baseline_all", None):
            out["cpu_baseline_all_cores"] = job.cpu_baseline_all()
    job.lib.close()
    # The other forms of the method, timed in the same run on the same GPU
    # (fewer steps): the table form of the same sample and K = 256 sets on
    # the tensor cores (4M events x 32 waves).
    if args.workload == "direct" and world == 1 and not args.no_secondary:
        sec = {}
        for name, make, steps in (
                ("table", lambda: job_direct(pwa, torch, stream, local, rank, form="table"), 300),
                ("tc", lambda: job_tc(pwa, torch, stream, local, rank, args.precision, gen="torch"), 40),
                ("direct_4M_32", lambda: job_direct32(pwa, torch, stream, local, rank), 200)):
            j = make()
            ms = measure(j, steps, 3, evict_l2, stream, None, rank, local, pwa, torch)
            sec[name] = {
                "workload": j.workload, "metric": getattr(j, "metric", METRIC),
                "value": j.evals_per_step * steps / (ms["total_ms"] / 1e3),
                "unit": getattr(j, "unit", UNIT), "steps": steps, "warmup": 3,
                "ms_per_step": ms["total_ms"] / steps, "dtype": j.dtype,
                "roofline": roofline(j, ms["total_ms"] / steps / 1e3, peaks),
                "e2e": {"value": j.evals_per_step * steps / ms["e2e_s"],
                        "unit": getattr(j, "unit", UNIT), "h2d_bytes_per_step": j.h2d,
                        "d2h_bytes_per_step": j.d2h},
                "gpu_launches": j.launches_per_step * steps, "status": ms["status"],
                "outputs_finite": ms["finite"],
                "config": dict(j.config, l2="flushed between timed steps" if j.flush
                               else "inputs larger than L2 (129 MB), no flush",
                               ms_per_step_back_to_back=ms["b2b_ms"])}
            if ms["clocks"] is not None:
                sec[name]["clocks"] = ms["clocks"]
            out["gpu_launches"] += j.launches_per_step * steps
            j.lib.close()
            del j
            torch.cuda.empty_cache()
        # the batched form against the plain single-fit form on the same
        # sample and GPU (parameter sets per second; accuracy of each against
        # the oracle: the tests' bounds, 4e-3 at 1M events for BFP16 and 1e-3
        # for the FP32 direct form)
        if "tc" in sec and "direct_4M_32" in sec:
            sec["tc"]["speedup_vs_direct_same_sample"] = sec["tc"]["value"] / sec["direct_4M_32"]["value"]
        out["secondary"] = sec
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def measure(job, steps, warmup, evict_l2, stream, dist, rank, local, pwa, torch):
    """Device-timed steps (CUDA events on the launching stream, L2 flushed
    before each where the job asks), back-to-back steps, and end-to-end host
    calls, with the clocks sampled during the timed steps."""
    for i in range(warmup):
        if job.flush:
            evict_l2(i)
        job.step()
    torch.cuda.synchronize()
    assert job.sync() in (pwa.PWA_OK,), "warm-up status"

    # raw nvidia-smi samples of the timed region (summarised into the line)
    clock_path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                              "bench_clocks_rank%d_%s.csv" % (rank, job.name))
    sampler = start_clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        if job.flush:
            evict_l2(i)                  # untimed
        starts[i].record(stream)
        job.step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    status = job.sync()
    finite = outputs_finite(job)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # back-to-back (no flush), for reference only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = max(3, steps // 2)
    e0.record(stream)
    for _ in range(nb):
        job.step()
    e1.record(stream)
    torch.cuda.synchronize()
    b2b_ms = e0.elapsed_time(e1) / nb
    # end to end through the public host call
    for _ in range(3):
        job.host_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        job.host_step()
    e2e_s = time.perf_counter() - t0
    clocks = None
    if sampler:
        sampler.terminate()
        sampler.wait()
        clocks = summarise_clocks(clock_path, local)
    return {"total_ms": total_ms, "b2b_ms": b2b_ms, "e2e_s": e2e_s, "status": status,
            "clocks": clocks, "finite": finite}


def roofline(job, avg_s, peaks):
    """The dominant kernel against its roofline, from the average step time."""
    if job.roof["bound"] == "hbm":
        achieved = job.roof["bytes"] / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm"], "unit": "GB/s",
                "frac": achieved / peaks["hbm"], "algorithmic_bytes_per_launch": job.roof["bytes"],
                "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": achieved / HBM_NOMINAL_GBS}
        if "flops" in job.roof:   # a contraction below the machine balance: tensor use for context
            tf = job.roof["flops"] / avg_s / 1e12
            roof.update({"tensor_achieved_tflops": tf, "tensor_frac": tf / peaks["bf16"]})
    elif job.roof["bound"] == "alu":
        achieved = job.roof["flops"] / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_NOMINAL_TFLOPS, "algorithmic_flops_per_step": job.roof["flops"],
                "peak_note": "nominal FP64 rate of the part (not measured); FP64 operations as "
                             "counted per event in config.flops_per_event"}
    else:
        achieved = job.roof["flops"] / avg_s / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16"], "algorithmic_flops_per_step": job.roof["flops"],
                "peak_nominal": BF16_NOMINAL_TFLOPS, "frac_nominal": achieved / BF16_NOMINAL_TFLOPS,
                "peak_note": "bf16 burst; the step time includes the small prep and final kernels"}
    roof.update({"traffic": TRAFFIC[job.name], "kernel": KERNELS[job.name],
                 "peak_kind": "nominal" if job.roof["bound"] == "alu" else peaks["kind"]})
    return roof

if __name__ == "__main__":
    main()
