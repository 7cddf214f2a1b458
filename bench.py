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

The headline form is BF16 (tensor-core hidden layers); the FP32 and FP8 forms of
the same step are timed on the same catalog afterwards and reported under
"forms" (with the BF16 / FP32 ratio).

--impl reference times the FP64 oracle (the CPU restatement of the method) on a
bounded sample of the same workload on this host's cores.
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
def build_workload(wid: int):
    from paper_2508_12117_gb300 import synth
    t = time.time()
    cat = synth.make_catalog(wid)
    return cat, time.time() - t


def launches_per_step(whiten: bool) -> int:
    # selection + pair table 5, travel times 1, residuals 1, whitening (CSR
    # assembly 4, components 15, work list 2, solvers 3 + merge 1), scatter/update 5
    return 5 + 1 + 1 + (26 if whiten else 0) + 5


# DRAM bytes (read + write) per unique pair of the BF16 tensor-core MLP kernel, from
# one ncu capture of the 100k-event step (8.42 MB read, 0.06 MB written, for about
# 0.372 M pairs; profiles/k_tt_mlp_tc_bf16_100kev.md); scaled by the pairs of a
# launch.  Only valid while that kernel is unchanged.
MLP_BF16_DRAM_BYTES_PER_PAIR = (8.423168e6 + 0.060160e6) / 372371.5


def flops_per_pair(H: int) -> float:
    # forward 3 H x H layers + 6 -> H + H -> 1, reverse 3 H x H layers + H -> 3
    return 12.0 * H * H + 20.0 * H


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    from paper_2508_12117_gb300 import binding, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cat, t_gen = build_workload(args.workload)
    prec = {"fp32": binding.FP32, "bf16": binding.BF16, "fp8": binding.FP8}[args.precision]
    h = cat.spec.hyper
    stream = torch.cuda.Stream()
    t0 = time.time()
    cfg = binding.config_for_catalog(cat, precision=prec, chain=rank, thin=1, sample_cap=1)
    ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations,
                          binding.net_for_catalog(cat), cfg, stream=stream.cuda_stream)
    t_create = time.time() - t0
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
    pairs = nobs = iters = 0
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + args.warmup + s)
        tm = ctx.spider_last_timing()      # waits for the step's events
        stage += np.array(tm["ms"])
        pairs += tm["pairs"]; nobs += tm["n_obs"]; iters += tm["pcg_iters"]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    # second timed pass, stage timers off (the step runs as one captured CUDA
    # graph) and no per-step host reads: the device throughput
    ctx.spider_set_timing(False)
    ctx.spider_sgld_step(eps, seed0 + 9_999)        # capture + first launch, untimed
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + 10_000 + s)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_dev = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ctx.spider_sync()
    # end to end through the public API: step + read the new state back to the host
    th_buf = None
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + 20_000 + s)
        th_buf, _ = ctx.spider_get_state()
    t_e2e = time.perf_counter() - t_e2e
    ms_dev, ms_total, e2e_ms = max_over_ranks([ms_dev, ms_total, t_e2e * 1e3], world)
    ctx.close()
    # the other precision forms on the same catalog (graph pass, same seeds)
    forms = {}
    if not args.no_forms:
        for other in ("fp32", "bf16", "fp8"):
            if other == args.precision:
                continue
            forms[other] = time_form(cat, other, eps, seed0, args, stream, world)
    if rank != 0:
        return None
    K = args.steps
    n_per_step = nobs / K
    p_per_step = pairs / K
    mlp_ms = stage[1] / K
    H = cat.spec.hidden
    pk, which = peaks()
    achieved = p_per_step * flops_per_pair(H) / (mlp_ms * 1e-3) / 1e12 if H else None
    if args.precision == "fp32":
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # FP32 FMA pipes at the maximum clock
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "k_tt_mlp_fp32<256>", "peak_source": "152 SMs x 128 FP32 lanes x 2 x max clock"}
    else:
        peak = pk["bf16_tflops_sustained"] * (2.0 if args.precision == "fp8" else 1.0)
        traffic = (MLP_BF16_DRAM_BYTES_PER_PAIR * p_per_step
                   if args.precision == "bf16" and args.workload in (3, 4) else None)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": "k_tt_mlp_tc",
                "peak_source": (f"bf16 sustained x 2 (nominal fp8/bf16 dense ratio), {which}"
                                if args.precision == "fp8" else f"bf16 sustained, {which}")}
    steps_s = replica_rate(world, K, ms_dev)
    state_bytes = cat.M * 16
    line = {
        "metric": METRIC, "value": steps_s, "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_dev / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": cat.spec.name, "events": cat.M, "stations": cat.S, "dd_obs": cat.N,
                   "minibatch_obs": h.batch_n, "block_obs": h.block_obs, "mlp": f"6-4x{H}-1",
                   "precision": args.precision, "l2": "inputs larger than L2 (3.2 GB tables, "
                   "fresh random blocks every step)", "parallelism": f"replicas x{world}"},
        "dd_obs_per_s": world * n_per_step * K / (ms_dev * 1e-3),
        "pairs_per_step": p_per_step, "whitening_iters_per_step": iters / K,
        "stage_ms_per_step": {"select_pairs": stage[0] / K, "travel_time_mlp": stage[1] / K,
                              "residual_whitening": stage[2] / K, "scatter_update": stage[3] / K,
                              "with_host_reads_ms_per_step": ms_total / K},
        "roofline": roof,
        "e2e": {"value": replica_rate(world, K, e2e_ms), "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": state_bytes,
                "note": "spider_sgld_step (eps, seed passed by value) + spider_get_state per step"},
        "forms": dict(forms, **({"bf16_over_fp32": steps_s / forms["fp32"]["value"]}
                                if args.precision == "bf16" and "fp32" in forms else {})),
        "gpu_launches": launches_per_step(cat.spec.hyper.kappa > 0) * K,
        "clocks": clk,
        "setup_s": {"generate": t_gen, "create": t_create},
    }
    return line


def time_form(cat, prec_name, eps, seed0, args, stream, world):
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
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + args.warmup + s)
        mlp += ctx.spider_last_timing()["ms"][1]
    ctx.spider_set_timing(False)
    ctx.spider_sgld_step(eps, seed0 + 9_999)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in range(args.steps):
        ctx.spider_sgld_step(eps, seed0 + 10_000 + s)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks([ev0.elapsed_time(ev1)], world)[0]
    ctx.close()
    K = args.steps
    return {"value": replica_rate(world, K, ms), "unit": "steps/s",
            "ms_per_step": ms / K, "travel_time_mlp_ms": mlp / K}


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
            "config": {"workload": "16 catalogs (1k-200k events, log-uniform) x 4 chains",
                       "events": sum(c.M for c in cats) * chains, "dd_obs": sum(c.N for c in cats) * chains,
                       "minibatch_obs_per_catalog": h.batch_n, "mlp": "6-4x128-1",
                       "l2": "inputs larger than L2"},
            "sequential": {"value": n_sub * 1e3 / ms_seq, "ms_per_round": ms_seq,
                           "note": "each sampler in its own context, stepped one after another"},
            "speedup_vs_sequential": ms_seq / ms_batch, "graph": info["graph"], "tuning": list(knobs),
            "tuning_ms": {k: v * 1e3 for k, v in tunings.items()}, "clocks": clk,
            "setup_s": {"generate": t_gen, "create": t_create}}


# ---------------------------------------------------------------- oracle timing
def oracle_sample(args, steps=3):
    """Time the FP64 oracle on a bounded sample of the workload: a catalog drawn
    with the same recipe at 1/50 of the events, minibatches of 2^14 observations;
    extrapolated linearly in observations and events to one full step."""
    from oracle import spider_oracle as O
    from paper_2508_12117_gb300 import synth
    full = synth.spec(args.workload)
    n_ev = max(2000, full.n_events // 50)
    sub = synth.scaled_spec(args.workload, n_ev, batch_n=1 << 14)
    cat = synth.make_catalog(sub)
    P = O.problem_from_catalog(cat)
    theta = cat.init_xyzt.copy()
    t_obs = 0.0
    t_ev = 0.0
    for s in range(steps):
        t = time.perf_counter()
        sel = P.batch(100 + s)
        _, g, _ = O.log_posterior(P, theta, sel)
        t_obs += time.perf_counter() - t
        t = time.perf_counter()
        eta = O.langevin_noise(P.M, 100 + s)
        theta = O.sgld_update(theta, g, full.hyper.eps, eta)
        t_ev += time.perf_counter() - t
    n_full = full.hyper.batch_n if full.hyper.batch_n else 1
    per_step = (t_obs / steps) * (n_full / (1 << 14)) + (t_ev / steps) * (full.n_events / P.M)
    return {"value": 1.0 / per_step, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle steps on a {P.M}-event / {P.N}-obs catalog of the same "
                      f"recipe with 2^14-obs minibatches, extrapolated linearly to 2^22 obs and "
                      f"{full.n_events} events per step"}, t_obs + t_ev


def run_reference(args, rank, world):
    if rank != 0:
        return None
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    base, secs = oracle_sample(args, steps=max(1, min(args.steps, 3)))
    return {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / base["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": synth_name(args.workload)},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


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
        if line is not None and not args.no_cpu_baseline:
            base, _ = oracle_sample(args)
            line["cpu_baseline"] = base
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
