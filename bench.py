"""Throughput of the SPIDER SGLD step on GB300 (one JSON line on rank 0).

Workload (default): the 1M-event catalog -- 1,000,000 events on 500 synthetic
faults, 200 stations, 200M dd observations, travel-time MLP 6 -> 4 x 256 SiLU -> 1,
minibatches of 2^22 observations (whole blocks of 4096), whitened likelihood.
A "step" is one full SGLD step: block selection, pair table, MLP forward + source
Jacobian for every touched pair, residuals, whitening solve, scatter, priors,
Langevin update.  Inputs (the 3.2 GB catalog tables) are resident in HBM and far
larger than L2; each step reads a fresh random 2% of them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8]
                  [--impl ours|reference] [--workload 4|3|2|1|5] [--no-forms]
                  [--no-cpu-baseline] [--scale-events N]

The headline form is BF16 (tensor-core hidden layers); the FP32 and FP8 forms of
the same step are timed on the same catalog afterwards and reported under
"forms" (with the BF16 / FP32 ratio).

--impl reference runs the FP64 oracle (the CPU restatement of the method) as an
SGLD chain on the same workload on this host's cores: warm-up, then up to K full
steps within a fixed time budget (a full oracle step of the 1M-event workload
takes ~20 s), reporting the steps it ran.  The line's cpu_baseline times one
full oracle step, or ~2 s of steps after a warm-up where a step is short
(rank 0, one GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SGLD steps/s (1M-event catalog, 2^22-obs minibatch)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return FALLBACK, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- replicas
def max_over_ranks(values, world):
    """Element-wise maximum over the ranks (the slowest replica sets the time)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def replica_rate(world, steps, ms):
    """Whole-job steps/s: every replica ran `steps` steps within `ms`."""
    return world * steps / (ms * 1e-3)


# ---------------------------------------------------------------- workload
def build_workload(wid: int, scale_events: int = 0):
    """The workload's catalog, or (scale_events > 0) a smaller catalog drawn
    with the same recipe (fault density, neighbours, stations per event) and
    minibatches covering the same fraction of it."""
    from paper_2508_12117_gb300 import synth
    t = time.time()
    if scale_events > 0:
        s = synth.spec(wid)
        bn = s.hyper.batch_n
        if bn > 0:
            bn = max(s.hyper.block_obs, int(bn * scale_events / s.n_events) // s.hyper.block_obs * s.hyper.block_obs)
        cat = synth.make_catalog(synth.scaled_spec(wid, scale_events, batch_n=bn))
    else:
        cat = synth.make_catalog(wid)
    return cat, time.time() - t


# DRAM bytes (read + write) per unique pair of the BF16 tensor-core MLP kernel, from
# one ncu capture of a 100k-event catalog of the 1M-event recipe (4.42 MB read,
# 0.8 KB written, for about 0.160 M pairs; profiles/k_tt_mlp_tc_bf16_100kev.md);
# scaled by the pairs of a launch.  Only valid while that kernel is unchanged.
MLP_BF16_DRAM_BYTES_PER_PAIR = (4.421632e6 + 768.0) / 160303.5


def flops_per_pair(H: int) -> float:
    # forward 3 H x H layers + 6 -> H + H -> 1, reverse 3 H x H layers + H -> 3
    return 12.0 * H * H + 20.0 * H


def hbm_bytes(n_obs, q_nodes, p_u, M, touched, pairs_per_event, sampled):
    """Algorithmic DRAM bytes per launch of the HBM-bound step kernels (every
    array element the kernel must read or write once):
      k_resid   20 B per observation (packed local indices, reduced dt, sqrt w,
                the residual written, two half-edge codes) + 47 B per local node
                (unique index, T hi/lo, pair, event, origin time, half-edge
                start, multi flag, u hi/lo, diagonal, row length, row offset);
      k_final   20 B per observation (indices, sqrt w, residual, q written,
                half-edge codes) + 19 B per local node (unique index, z hi/lo,
                half-edge start, multi flag, node sum written);
      k_merge_s 61 B per unique pair (occurrence, pair, event, sub-problem,
                multi flag, node sum, Jacobian, contribution written, 2 stamps);
      k_event   44 B per event (sub-problem, stamp, state read and written,
                noise counter) + 16 B per event when a sample is stored, plus per
                touched event its pair range and stamps (8 + 4 per pair) and
                16 B per pair contribution."""
    return {
        "k_resid": 20.0 * n_obs + 47.0 * q_nodes,
        "k_final": 20.0 * n_obs + 19.0 * q_nodes,
        "k_merge_s": 61.0 * p_u,
        "k_event": (44.0 + (16.0 if sampled else 0.0)) * M + touched * (8.0 + 4.0 * pairs_per_event)
        + 16.0 * p_u,
    }


def measure_fp8_peak():
    """Dense E4M3 x E4M3 -> BF16 GEMM throughput of cuBLASLt (torch._scaled_mm),
    8192^3, best of 10 timed with CUDA events: the FP8 denominator measured on
    this GPU.  None when the call is unavailable."""
    import torch
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    except Exception:
        return None


def peak_for(clk, pk):
    """BF16 denominator: the burst figure unless the clock record shows the power
    cap or an SM clock well below its maximum during the timed region."""
    capped = "sw_power_cap" in (clk.get("reasons") or [])
    mhz, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz") or pk.get("sm_max_mhz", 2070.0)
    low = mhz is not None and mx and mhz < 0.95 * mx
    if capped or low:
        return pk["bf16_tflops_sustained"], "bf16 sustained"
    return pk["bf16_tflops"], "bf16 burst"


def host_cpu():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        if not model:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    from paper_2508_12117_gb300 import binding, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cat, t_gen = build_workload(args.workload, args.scale_events)
    prec = {"fp32": binding.FP32, "bf16": binding.BF16, "fp8": binding.FP8}[args.precision]
    h = cat.spec.hyper
    l2_resident = cat.N * 12 <= 129e6          # observation tables (12 B per obs) within the 129 MB L2
    stream = torch.cuda.Stream()
    t0 = time.time()
    cfg = binding.config_for_catalog(cat, precision=prec, chain=rank, thin=1, sample_cap=1)
    ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations,
                          binding.net_for_catalog(cat), cfg, stream=stream.cuda_stream)
    t_create = time.time() - t0
    info = ctx.spider_info()
    eps = h.eps
    seed0 = 1_000_003 * (rank + 1)
    ctx.spider_set_timing(True)
    for w in range(args.warmup):
        ctx.spider_sgld_step(eps, seed0 + w)
    ctx.spider_sync()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.5)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = np.zeros(5)
    kern, wphase = {}, {}
    pairs = nobs = iters = touched = 0
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + args.warmup + s)
        tm = ctx.spider_last_timing()      # waits for the step's events
        kt, te = ctx.spider_last_kernel_timing()
        wt = ctx.spider_last_whiten_timing()
        stage += np.array(tm["ms"])
        for k_, v_ in kt.items():
            kern[k_] = kern.get(k_, 0.0) + v_
        for k_, v_ in wt.items():
            wphase[k_] = wphase.get(k_, 0.0) + v_
        pairs += tm["pairs"]; nobs += tm["n_obs"]; iters += tm["pcg_iters"]; touched += te
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    # second timed pass, stage timers off (the step runs as one captured CUDA
    # graph) and no per-step host reads: the device throughput
    ctx.spider_set_timing(False)
    ctx.spider_sgld_step(eps, seed0 + 9_999)        # capture + first launch, untimed
    torch.cuda.synchronize()
    graph_kernels = ctx.spider_info()["graph_kernels"]      # kernel nodes of the step graph
    # inputs that fit in L2 (small workloads): L2 flushed before every timed step
    ms_dev = timed_graph_steps(ctx, eps, seed0 + 10_000, args.steps, stream, l2_resident)
    clk = clocks.stop()
    ctx.spider_sync()
    # end to end through the public API: step + read the new state back into a
    # page-locked host buffer (the caller's), every step
    host_state = torch.empty((cat.M, 4), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + 20_000 + s)
        ctx.spider_get_state(out_ptr=host_state.data_ptr())
    t_e2e = time.perf_counter() - t_e2e
    ms_dev, ms_total, e2e_ms = max_over_ranks([ms_dev, ms_total, t_e2e * 1e3], world)
    ctx.close()
    # the other precision forms on the same catalog (graph pass, same seeds)
    forms = {}
    pk, which = peaks()
    if not args.no_forms and cat.spec.forward == "mlp":
        for other in ("fp32", "bf16", "fp8"):
            if other == args.precision:
                continue
            forms[other] = time_form(cat, other, eps, seed0, args, stream, world, clk, pk)
    if rank != 0:
        return None
    K = args.steps
    n_per_step = nobs / K
    p_per_step = pairs / K
    mlp_ms = stage[1] / K
    H = cat.spec.hidden
    kms = {k_: v_ / K for k_, v_ in kern.items()}
    roof = mlp_roofline(args.precision, H, p_per_step, mlp_ms, clk, pk, which,
                        args.workload in (3, 4), measure_fp8_peak() if args.precision == "fp8" else None)
    # HBM-bound kernels: algorithmic bytes per launch / their CUDA-event time
    q_sel = info["local_nodes"] * n_per_step / max(1, info["obs"])
    nb = hbm_bytes(n_per_step, q_sel, p_per_step, cat.M, touched / K, info["pairs"] / cat.M, True)
    hbm = {}
    for kname, byt in nb.items():
        ms = kms.get(kname, 0.0)
        if ms > 0:
            ach = byt / (ms * 1e-3) / 1e9
            hbm[kname] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                          "frac": ach / pk["hbm_gbs"], "bytes": byt, "ms": ms, "traffic": None}
    steps_s = replica_rate(world, K, ms_dev)
    state_bytes = cat.M * 32
    line = {
        "metric": METRIC if args.workload == 4 and not args.scale_events else f"SGLD steps/s ({cat.spec.name})",
        "value": steps_s, "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_dev / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": cat.spec.name, "events": cat.M, "stations": cat.S, "dd_obs": cat.N,
                   "minibatch_obs": h.batch_n, "block_obs": h.block_obs,
                   "mlp": f"6-4x{H}-1" if H else "analytic homogeneous",
                   "precision": args.precision,
                   "l2": ("inputs larger than L2 (tables of the catalog, fresh random blocks every step)"
                          if not l2_resident else
                          "inputs smaller than L2: L2 flushed (256 MB written) before every timed step, "
                          "outside the timed intervals"),
                   "parallelism": f"replicas x{world}"},
        "dd_obs_per_s": world * n_per_step * K / (ms_dev * 1e-3),
        "pairs_per_step": p_per_step, "touched_events_per_step": touched / K,
        "whitening_iters_per_step": iters / K,
        "stage_ms_per_step": {"select_pairs": stage[0] / K, "travel_time_mlp": stage[1] / K,
                              "residual_whitening": stage[2] / K, "scatter_update": stage[3] / K,
                              "with_host_reads_ms_per_step": ms_total / K},
        "kernel_ms_per_step": kms,
        "whitening_phases_ms_per_step": {k_: v_ / K for k_, v_ in wphase.items()},
        "roofline": roof,
        "roofline_hbm": hbm,
        "e2e": {"value": replica_rate(world, K, e2e_ms), "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": state_bytes,
                "note": "spider_sgld_step (eps, seed passed by value) + spider_get_state into a "
                        "page-locked host buffer (M x 4 FP64) per step"},
        "forms": dict(forms, **({"bf16_over_fp32": steps_s / forms["fp32"]["value"]}
                                if args.precision == "bf16" and "fp32" in forms else {})),
        "gpu_launches": graph_kernels * K,
        "clocks": clk,
        "setup_s": {"generate": t_gen, "create": t_create},
    }
    line["_cat"] = cat
    return line


def mlp_roofline(prec, H, p_per_step, mlp_ms, clk, pk, which, traffic_ok, fp8_peak):
    if not H or mlp_ms <= 0:
        return {"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "kernel": "k_tt_homogeneous",
                "note": "analytic travel times: the step is bound by launch latency"}
    achieved = p_per_step * flops_per_pair(H) / (mlp_ms * 1e-3) / 1e12
    if prec == "fp32":
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # FP32 FMA pipes at the maximum clock
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": f"k_tt_mlp_fp32<{H}>",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max clock"}
    if prec == "fp8":
        if fp8_peak:
            peak, src = fp8_peak, "fp8 e4m3 cuBLASLt GEMM 8192^3 measured in this run (burst)"
        else:
            b, _ = peak_for(clk, pk)
            peak, src = 2.0 * b, "bf16 measured x 2 (nominal fp8/bf16 dense ratio)"
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": f"k_tt_mlp_tc<{H},1>", "peak_source": src}
    peak, src = peak_for(clk, pk)
    traffic = MLP_BF16_DRAM_BYTES_PER_PAIR * p_per_step if traffic_ok else None
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": f"k_tt_mlp_tc<{H},0>",
            "peak_source": f"{src}, {which}"}


def timed_graph_steps(ctx, eps, seed_base, K, stream, flush_l2):
    """Device ms of K graph steps on `stream` (CUDA events).  flush_l2: write a
    256 MB buffer before every step, outside the timed intervals, and add up the
    steps; otherwise one interval around all K steps."""
    import torch
    if flush_l2:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        ms = 0.0
        for s in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(s & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.spider_sgld_step(eps, seed_base + s)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(K):
        ctx.spider_sgld_step(eps, seed_base + s)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def time_form(cat, prec_name, eps, seed0, args, stream, world, clk, pk):
    """Steps/s of another precision form of the same step on the same catalog:
    warm-up, then K steps of the captured graph timed with CUDA events."""
    import torch
    from paper_2508_12117_gb300 import binding
    prec = {"fp32": binding.FP32, "bf16": binding.BF16, "fp8": binding.FP8}[prec_name]
    cfg = binding.config_for_catalog(cat, precision=prec, chain=0, thin=1, sample_cap=1)
    ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations,
                          binding.net_for_catalog(cat), cfg, stream=stream.cuda_stream)
    ctx.spider_set_timing(True)
    for w in range(args.warmup):
        ctx.spider_sgld_step(eps, seed0 + w)
    mlp = 0.0
    pairs = 0
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + args.warmup + s)
        tm = ctx.spider_last_timing()
        mlp += tm["ms"][1]
        pairs += tm["pairs"]
    ctx.spider_set_timing(False)
    ctx.spider_sgld_step(eps, seed0 + 9_999)
    torch.cuda.synchronize()
    ms = timed_graph_steps(ctx, eps, seed0 + 10_000, args.steps, stream, cat.N * 12 <= 129e6)
    ms = max_over_ranks([ms], world)[0]
    ctx.close()
    K = args.steps
    roof = mlp_roofline(prec_name, cat.spec.hidden, pairs / K, mlp / K, clk, pk, "measured", False,
                        measure_fp8_peak() if prec_name == "fp8" else None)
    return {"value": replica_rate(world, K, ms), "unit": "steps/s",
            "ms_per_step": ms / K, "travel_time_mlp_ms": mlp / K, "roofline": roof}


# ---------------------------------------------------------------- batched
def run_batched(args, rank, world):
    """16 catalogs of uneven sizes x 4 chains advanced together (one CUDA graph
    per step) against the same 64 samplers stepped one context at a time."""
    import torch
    from paper_2508_12117_gb300 import autotune, binding, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t = time.time()
    specs = synth.batch_specs(16)
    cats = [synth.make_catalog(s) for s in specs]
    t_gen = time.time() - t
    chains = 4
    prec = {"fp32": binding.FP32, "bf16": binding.BF16, "fp8": binding.FP8}[args.precision]
    net = binding.Net(binding.TT_MLP, mlp=synth.batch_network())
    h = specs[0].hyper
    cfg = binding.make_config(sigma=h.sigma, kappa=h.kappa, p=h.p, ell=h.ell, eps_w=h.eps_w,
                              sig_e=h.sig_e, sig_c=h.sig_c, batch_n=h.batch_n, block_obs=h.block_obs,
                              precision=prec, thin=1, sample_cap=1)
    stream = torch.cuda.Stream()
    t = time.time()
    bat = binding.Context.batch(cats, chains, net, cfg, stream=stream.cuda_stream)
    t_create = time.time() - t
    knobs, tunings = autotune.autotune(bat, h.eps, prec, 128, use_cache=False)
    for w in range(args.warmup):
        bat.spider_sgld_step(h.eps, 700 + w)
    bat.spider_sync()
    info = bat.spider_info()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in range(args.steps):
        bat.spider_sgld_step(h.eps, 800 + s)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_batch = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    bat.close()
    # the same samplers one context at a time (chain 0 of each catalog; 4 chains cost 4x)
    ms_seq = 0.0
    for ci, cat in enumerate(cats):
        c1 = binding.make_config(sigma=h.sigma, kappa=h.kappa, p=h.p, ell=h.ell, eps_w=h.eps_w,
                                 sig_e=h.sig_e, sig_c=h.sig_c, batch_n=h.batch_n, block_obs=h.block_obs,
                                 precision=prec, catalog=ci, thin=1, sample_cap=1)
        ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations, net, c1,
                              stream=stream.cuda_stream)
        for w in range(2):
            ctx.spider_sgld_step(h.eps, 900 + w)
        torch.cuda.synchronize()
        ev0.record(stream)
        for s in range(args.steps):
            ctx.spider_sgld_step(h.eps, 1000 + s)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_seq += chains * ev0.elapsed_time(ev1) / args.steps
        ctx.close()
    n_sub = len(cats) * chains
    return {"metric": "aggregate SGLD steps/s, 16 catalogs x 4 chains in one context",
            "value": n_sub * 1e3 / ms_batch, "unit": "sub-problem steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": f"{len(cats)} catalogs ({min(c.M for c in cats)}-{max(c.M for c in cats)} "
                                   f"events, drawn log-uniform in 1k-200k) x {chains} chains",
                       "events": sum(c.M for c in cats) * chains, "dd_obs": sum(c.N for c in cats) * chains,
                       "minibatch_obs_per_catalog": h.batch_n, "mlp": "6-4x128-1",
                       "l2": "inputs larger than L2"},
            "sequential": {"value": n_sub * 1e3 / ms_seq, "ms_per_round": ms_seq,
                           "note": "each sampler in its own context, stepped one after another"},
            "speedup_vs_sequential": ms_seq / ms_batch, "graph": info["graph"], "tuning": list(knobs),
            "gpu_launches": info["graph_kernels"] * args.steps,
            "tuning_ms": {k: v * 1e3 for k, v in tunings.items()}, "clocks": clk,
            "setup_s": {"generate": t_gen, "create": t_create}}


# ---------------------------------------------------------------- oracle timing
def oracle_step(cat, seed):
    """Time the FP64 oracle on real steps of the workload: the same catalog,
    the minibatch each step's seed selects (all of it), the log-posterior
    gradient, the Langevin noise and the update.  The oracle's one-time set-up
    (canonical order, edge weights) is timed apart and not counted.  A step
    that takes under 2 s counts as a warm-up and the next steps, up to about
    2 s of them, are timed instead; a longer one is the sample itself.
    Returns (cpu_baseline entry, seconds per timed step)."""
    from oracle import spider_oracle as O
    t = time.perf_counter()
    P = O.problem_from_catalog(cat)
    t_setup = time.perf_counter() - t
    theta = cat.init_xyzt.copy()
    n = pairs = 0

    def one(sd):
        nonlocal theta, n, pairs
        t0 = time.perf_counter()
        sel = None if (P.batch_n <= 0 or P.batch_n >= P.N) else P.batch(sd)
        _, g, info = O.log_posterior(P, theta, sel)
        theta = O.sgld_update(theta, g, cat.spec.hyper.eps, O.langevin_noise(P.M, sd))
        n, pairs = info["n"], info["T"].shape[0]
        return time.perf_counter() - t0

    secs, steps, warm = one(seed), 1, 0
    if secs < 2.0:
        warm, secs, steps = 1, 0.0, 0
        while steps < 1000 and (steps == 0 or secs < 2.0):
            secs += one(seed + 1 + steps)
            steps += 1
    hc = host_cpu()
    per = secs / steps
    return {"value": 1.0 / per, "unit": "steps/s", "cores": hc["nproc"], "kind": "oracle",
            "cpu_model": hc["cpu_model"], "nproc": hc["nproc"], "steps": steps,
            "sample": (f"{steps} full oracle step(s) of this workload after {warm} untimed warm-up step(s) "
                       f"({P.M} events, {n} observations per minibatch, {pairs} travel-time pairs), not "
                       f"extrapolated; numpy elementwise work on 1 thread, BLAS matrix products on up to "
                       f"{hc['nproc']} threads; set-up {t_setup:.1f} s not counted")}, per


REFERENCE_BUDGET_S = 90.0      # wall time the reference arm's timed steps may take


def run_reference(args, rank, world):
    """The oracle's SGLD chain on the workload: up to --warmup untimed steps (at
    least one, none started after a sixth of REFERENCE_BUDGET_S), then up
    to --steps timed full steps, stopped after the first that ends past the
    budget; `warmup` and `steps` are the numbers actually run."""
    if rank != 0:
        return None
    from oracle import spider_oracle as O
    cat, t_gen = build_workload(args.workload, args.scale_events)
    t = time.perf_counter()
    P = O.problem_from_catalog(cat)
    t_setup = time.perf_counter() - t
    theta = cat.init_xyzt.copy()
    eps = cat.spec.hyper.eps
    n_obs = 0
    seed = 1_000_003 + 10_000

    def step():
        nonlocal theta, n_obs, seed
        sel = None if (P.batch_n <= 0 or P.batch_n >= P.N) else P.batch(seed)
        _, g, info = O.log_posterior(P, theta, sel)
        theta = O.sgld_update(theta, g, eps, O.langevin_noise(P.M, seed))
        n_obs = info["n"]
        seed += 1

    warm, t = 0, time.perf_counter()
    while warm < max(1, args.warmup) and time.perf_counter() - t < REFERENCE_BUDGET_S / 6:
        step()
        warm += 1
    steps, secs = 0, 0.0
    while steps < max(1, args.steps) and secs < REFERENCE_BUDGET_S:
        t = time.perf_counter()
        step()
        secs += time.perf_counter() - t
        steps += 1
    hc = host_cpu()
    value = steps / secs
    base = {"value": value, "unit": "steps/s", "cores": hc["nproc"], "kind": "oracle",
            "cpu_model": hc["cpu_model"], "nproc": hc["nproc"], "steps": steps,
            "sample": (f"{steps} full oracle step(s) of this workload ({P.M} events, {n_obs} observations "
                       f"per minibatch), not extrapolated; numpy elementwise work on 1 thread, BLAS "
                       f"matrix products on up to {hc['nproc']} threads; set-up {t_setup:.1f} s not counted")}
    metric = METRIC if args.workload == 4 and not args.scale_events else f"SGLD steps/s ({cat.spec.name})"
    return {"impl": "reference", "metric": metric, "value": value, "unit": "steps/s",
            "n_gpus": world, "steps": steps, "warmup": warm, "steps_requested": args.steps,
            "ms_per_step": secs / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cat.spec.name, "events": cat.M, "dd_obs": cat.N,
                       "minibatch_obs": cat.spec.hyper.batch_n},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": (f"the oracle's chain: {warm} untimed warm-up step(s), then {steps} of {args.steps} "
                     f"requested timed steps within a {REFERENCE_BUDGET_S:.0f} s budget; catalog "
                     f"generation {t_gen:.1f} s not counted")}


def synth_name(wid):
    from paper_2508_12117_gb300 import synth
    return synth.spec(wid).name


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--no-forms", action="store_true",
                    help="skip timing the other precision forms on the same catalog")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale-events", type=int, default=0,
                    help="a smaller catalog of the workload's recipe with this many events "
                         "(profiling captures; not a bench line)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == 5:
        line = run_batched(args, rank, world)
    else:
        line = run_ours(args, rank, world)
        if line is not None:
            cat = line.pop("_cat")
            if not args.no_cpu_baseline and world == 1:     # the oracle baseline: rank 0 at N = 1
                base, _ = oracle_step(cat, 1_000_003 + 10_000)
                line["cpu_baseline"] = base
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
