#!/usr/bin/env python
"""Throughput benchmark: BP + p-flip decoding of the 3D toric code.

Default workload (``bp_pflip_L32``): L = 32 (98,304 edge qubits), p = q = 4%,
BP with 16 FP32 iterations (measurement-error variables on) followed by 32
flip / p-flip applications cycling P F F P F F, 10^5 samples per GPU.  One
step = one code cycle through the public entry point ``toric3d_run_cycles``
(qubit noise, noisy measurement, BP, the schedule, and the logical readout of
the residual error).  The metric is decoded qubit-cycles per second over all
GPUs (3 L^3 x samples x cycles / time); every rank decodes its own disjoint
sample range (weak scaling, no data-path collective).

``--impl reference`` times the CPU oracle on a bounded sample of the same
workload instead.

Prints one JSON line (rank 0).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import toric3d_inputs as inp  # noqa: E402

METRIC = "qubit-cycles decoded/s at L=32 p=4%: BP+p-flip vs learned+p-flip, equal logical err"
# `value` is the BP + p-flip decoder (the decoder the reference arm times); the line's
# learned_pflip object holds learned + p-flip on the same workload and its ratio.
VALUE_IS = "BP+p-flip; learned_pflip.value = learned+p-flip, learned_pflip.vs_bp_pflip = their ratio"

# DRAM bytes (read + write) per edge-sample of the dominant kernel from one
# ncu capture of the current k_bp_step (L = 32, 1024 samples; traffic grows in
# proportion to the samples a launch covers, so it scales to full launches).
# Set to None when the kernel changes until it is captured again.
BP_STEP_TRAFFIC = {"first_iteration": 15.69, "full_iteration": 31.90}
# The same for k_flip_tiled inside the FFPFF cycle at p = q = 4% (L = 32, 8192 samples, the
# four flip applications of one cycle: 322.4 MB of DRAM traffic each on average, per
# qubit-sample 0.400 B against the dense 0.5 B: e is touched only where a word has a flipped
# lane, so the figure depends on the noise rates).  None when the kernel changes.
FLIP_TRAFFIC_P = 0.04
FLIP_TRAFFIC = 322.4e6 / (98304 * 8192)
UNIT = "qubit-cycles/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="bp_pflip_L32", choices=sorted(inp.WORKLOADS))
    ap.add_argument("--samples", type=int, default=0, help="samples per GPU (default: the workload's)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU baseline sample")
    ap.add_argument("--reference-seconds", type=float, default=60.0,
                    help="--impl reference: oracle time over all steps (default 60 s)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (default: as many as --steps, at least 3)")
    ap.add_argument("--e2e-parts", type=int, default=2,
                    help="end-to-end: sample ranges whose copies overlap the others' decoding")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned pre-decoder + p-flip leg of the same workload")
    ap.add_argument("--learned-chunk", type=int, default=16384,
                    help="samples per pre-decoder launch (bounds its activation workspace)")
    ap.add_argument("--fallback-sigmas", type=float, default=4.0,
                    help="learned leg: BP + p-flip fallback above q 3L^3 + this many sigma unsatisfied checks")
    return ap.parse_args()


def workload_config(w, S):
    return {"workload": w.name, "L": list(w.sizes), "qubits": sum(inp.n_bits(L) for L in w.sizes),
            "p": w.p, "q": w.q,
            "decoder": w.decoder, "bp_iters": w.bp_iters, "bp_meas_nodes": w.bp_meas_nodes,
            "schedule": w.schedule, "n_apply": w.n_apply, "samples_per_gpu": S,
            "cycles_per_step": 1, "T": w.T, "seed": w.seed,
            "l2": "inputs larger than L2 (state and BP messages are GBs)"}


# ------------------------------------------------------------------ CPU oracle leg
def _oracle_worker(args):
    L, p, q, seed, kw, sample0, count, cycle0 = args
    import oracle
    cfg = oracle.make_cfg(L, 1, p, q, seed, cycle0=cycle0, **kw)
    oracle.run_batch(cfg, sample0, count)
    return count


def oracle_kwargs(w):
    return dict(use_bp=w.decoder.startswith("bp"), bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes,
                schedule=w.schedule, n_apply=w.n_apply)


def time_oracle(w, budget_s, cycle0=0):
    """Time the oracle on one code cycle of a bounded number of samples of every
    lattice size of the workload, one process per host core (spawned, so no
    CUDA state is inherited)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    jobs, per_size = [], {}
    for L in w.sizes:
        cfg = oracle.make_cfg(L, 1, w.p, w.q, w.seed, **oracle_kwargs(w))
        t0 = time.perf_counter()
        oracle.run_batch(cfg, 0, 1)
        one = max(time.perf_counter() - t0, 1e-4)
        per_core = max(1, int(budget_s / len(w.sizes) / one))
        per_size[L] = per_core * cores
        jobs += [(L, w.p, w.q, w.seed, oracle_kwargs(w), 64 * 1024 * i, per_core, cycle0) for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        pool.map(_oracle_worker, jobs)
        dt = time.perf_counter() - t0
    value = sum(inp.n_bits(L) * k for L, k in per_size.items()) / dt
    sample = ", ".join(f"{k} samples at L={L}" for L, k in per_size.items())
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sample}, 1 code cycle each, {cores} processes", "seconds": dt}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = inp.WORKLOADS[args.workload]
    S = args.samples or w.n_samples
    budget = max(0.5, args.reference_seconds / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        time_oracle(w, budget / 4, cycle0=i)
    vals, secs, last = [], [], None
    for i in range(args.steps):
        last = time_oracle(w, budget, cycle0=args.warmup + i)
        vals.append(last["value"])
        secs.append(last["seconds"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "value_is": "BP+p-flip (the oracle)",
            "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox noise)",
            "config": dict(workload_config(w, S), parallelism=f"replicas{args.gpus}"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CUDA arm
# Algorithmic FLOPs of the pre-decoder per site and sample: three 3x3x3
# convolutions (6 -> 16, 16 -> 16, 16 -> 16 channels) and the 16 -> 3 head.
CNN_FLOP_PER_SITE = 2 * 27 * 16 * (6 + 16 + 16) + 2 * 16 * 3
# Tensor-core FLOPs the kernels execute per site and sample (2 x 2 columns of
# output sites; each MMA spans the TMEM columns an input tile reaches, zero
# blocks included): 168 weight blocks of 16 x 16 per input plane of a column
# (4 sites) and 128 samples in a hidden layer, 88 in the first (two sites per
# K = 16), each block 128 x 16 x 16 multiply-adds.
CNN_MMA_FLOP_PER_SITE = (88 + 168 + 168) * 2 * 128 * 16 * 16 / (4 * 128)
WEIGHTS = os.path.join(ROOT, "paper_2212_06985_gb300", "weights", "cnn_L12_p04.npz")


def bp_chunk(L, S):
    """BP chunk: 25,024 samples, fewer where the two message buffers (48 L^3 bytes per
    sample each) would pass 96 GB."""
    fit = int(48e9 // (48 * L ** 3)) // 64 * 64
    return max(64, min(S, 25024, fit))


def learned_chunk(L, S, cap):
    """Pre-decoder chunk: `cap` samples, fewer where its activations (80 B per site-sample)
    would pass 48 GB."""
    fit = int(48e9 // (80 * L ** 3)) // 128 * 128
    return max(128, min(S, cap, fit))


def learned_leg(args, t3d, w, S, sample0, dev, stream, barrier, world, peaks):
    """The same workload decoded by the learned pre-decoder + the same flip /
    p-flip schedule instead of BP (one cycle per step through toric3d_run_batch)."""
    import numpy as np
    import torch

    with np.load(WEIGHTS) as z:
        params = torch.from_numpy(np.array(z["params"], dtype=np.float32)).to(dev)
    blob = torch.empty(t3d.toric3d_cnn_blob_bytes(), dtype=torch.uint8, device=dev)
    t3d.toric3d_cnn_prepare(params, blob)
    sizes = w.sizes
    W = inp.words_for(S)
    states = [torch.zeros((inp.n_bits(L), W), dtype=torch.int64, device=dev) for L in sizes]
    prevs = [torch.zeros_like(e) for e in states]
    counts = [torch.zeros(8, dtype=torch.int64, device=dev) for _ in sizes]
    fallback = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in sizes]
    batch = t3d.make_batch([dict(L=L, n_samples=S, sample0=sample0, e=e, s_prev=sp, counts8=c, fallback_words=f)
                            for L, e, sp, c, f in zip(sizes, states, prevs, counts, fallback)])
    # BP + p-flip fallback for every 64-sample word in which a sample's decoded syndrome keeps
    # more unsatisfied checks than the noisy measurement alone leaves (q 3L^3 + k sigma)
    cfg = t3d.make_run_cfg(w.L, 1, w.p, w.q, w.seed, S, sample0=sample0, schedule=w.schedule, n_apply=w.n_apply,
                           bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes,
                           bp_chunk_samples=learned_chunk(max(sizes), S, args.learned_chunk), cnn_blob=blob,
                           fallback_max_weight=0, fallback_sigmas=args.fallback_sigmas)
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev)

    def step(t):
        cfg.cycle0 = t
        t3d.toric3d_run_batch(cfg, batch, work, stream=stream)

    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            step(t)
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    fb0 = sum(int(f.item()) for f in fallback)
    t3d.toric3d_profile_reset()
    t3d.toric3d_profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for t in range(args.warmup, args.warmup + args.steps):
            step(t)
        ev1.record(stream)
    ev1.synchronize()
    t3d.toric3d_profile_enable(False)
    t3d.toric3d_cnn_status()
    fb_timed = sum(int(f.item()) for f in fallback) - fb0
    prof = {k: t3d.toric3d_profile_read(k) for k in t3d.KERNEL_KINDS}
    t3d.toric3d_profile_reset()
    ms = ev0.elapsed_time(ev1)
    t_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms = float(t_max.item())
    qubits = sum(inp.n_bits(L) for L in sizes)
    sites = sum(L ** 3 for L in sizes)
    cnn_ms, cnn_launches = prof["cnn"]
    flop = CNN_FLOP_PER_SITE * sites * S * args.steps
    tf_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
    achieved = flop / (cnn_ms / 1e3) / 1e12 if cnn_ms > 0 else 0.0
    del work
    return {
        "decoder": "learned pre-decoder (3 x conv3d 3x3x3, 16 ch, BF16 tensor cores) + " + w.schedule + " x "
                   + str(w.n_apply), "weights": os.path.relpath(WEIGHTS, ROOT),
        "value": qubits * S * world * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
        "gpu_launches": sum(v[1] for v in prof.values()),
        "kernels_ms": {k: v[0] for k, v in prof.items() if v[1]},
        "roofline": {"kernel": "k_conv_col (3 layers) + k_expand_bits + k_dec_apply", "bound": "tensor",
                     "achieved": achieved, "peak": tf_peak, "unit": "TFLOP/s", "frac": achieved / tf_peak,
                     "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured)" if peaks
                     else "fallback 1.7 PFLOP/s sustained",
                     "algorithmic_flop_per_site_sample": CNN_FLOP_PER_SITE,
                     "executed_mma_tflops": CNN_MMA_FLOP_PER_SITE * sites * S * args.steps / (cnn_ms / 1e3) / 1e12
                     if cnn_ms > 0 else None,
                     "share_of_step": cnn_ms / ms if ms else None},
        "fallback": {"gate": f"fallback_max_weight 0 + fallback_sigmas {args.fallback_sigmas}: a word goes back to "
                             f"BP{w.bp_iters} + the schedule when a sample keeps more than q 3L^3 + "
                             f"{args.fallback_sigmas} sigma unsatisfied checks",
                     "thresholds": {str(L): int(math.floor(w.q * inp.n_bits(L) + args.fallback_sigmas *
                                                           math.sqrt(w.q * (1 - w.q) * inp.n_bits(L))))
                                    for L in sizes},
                     "words_per_step": fb_timed / args.steps,
                     "word_fraction": fb_timed / (args.steps * W * len(sizes))},
        "logical_counts": [c.cpu().tolist() for c in counts],
        "logical_counts_after_cycles": args.warmup + args.steps,
        "chunk_samples": learned_chunk(max(sizes), S, args.learned_chunk),
    }


# Flip / p-flip cycles.  Algorithmic bytes per qubit-sample of one launch of each
# kernel kind: noise reads and writes e (0.25 B); the measurement reads e and
# writes s (0.25 B); a flip application reads s and e and writes both (0.5 B);
# a p-flip application (decision pass + syndrome pass) also writes and reads
# the flip words (0.875 B).
SWEEP_BYTES = {"noise": 0.25, "syndrome": 0.25, "flip": 0.5, "pflip": 0.875}
# Warp instructions per 64-sample word of each qubit (noise), check (syndrome)
# or site (the decision pass of one p-flip application) at p = q = 4%, from one
# ncu capture of the current kernels (smsp__inst_executed.sum / (units x words),
# L = 32, 8192 samples: 157.0 M, 189.7 M and 51.8 M instructions).  The Philox
# arithmetic binds these kernels on the instruction issue rate.
SWEEP_INST_P = 0.04
SWEEP_INST = {"noise": 157.0e6 / (98304 * 128), "syndrome": 189.7e6 / (98304 * 128), "pflip": 51.8e6 / (32768 * 128)}
# The p-flip syndrome pass reads the flip words and updates s in place (0.375 B).
PFLIP_APPLY_BYTES = 0.375


def sweep_roofline(prof, w, qubits, S, steps, ms, hbm_peak, peak_source, clk):
    """Roofline of the dominant kernel of a flip / p-flip cycle: HBM for the flip
    application, the instruction-issue rate (152 SMs x 4 schedulers x 1 warp
    instruction per clock at the sampled SM clock) for the Philox-bound kernels
    once their instruction counts are known; the whole cycle's HBM fraction beside."""
    n_p = sum(1 for k in range(w.n_apply) if w.schedule[k % len(w.schedule)] == "P")
    per_step = {"noise": 1, "syndrome": 1, "flip": w.n_apply - n_p, "pflip": n_p}
    kinds = {k: prof[k] for k in SWEEP_BYTES if prof[k][1]}
    dom = max(kinds, key=lambda k: kinds[k][0])
    d_ms, d_launches = kinds[dom]
    apps = per_step[dom] * steps                      # applications (a p-flip one is two launches)
    t_app = d_ms / apps / 1e3
    words = (S + 63) // 64
    cycle_bytes = sum(SWEEP_BYTES[k] * per_step[k] for k in SWEEP_BYTES) * qubits * S * steps
    out = {"kernel": {"noise": "k_noise", "syndrome": "k_syndrome", "flip": "k_flip_tiled",
                      "pflip": "k_pflip_decide + k_pflip_apply"}[dom],
           "launches": d_launches, "avg_launch_ms": d_ms / d_launches, "ms_per_application": 1e3 * t_app,
           "share_of_step": d_ms / ms, "cycle_hbm_frac": cycle_bytes / (ms / 1e3) / 1e9 / hbm_peak,
           "kernels_hbm_frac": {k: SWEEP_BYTES[k] * qubits * S * steps * per_step[k] / (v[0] / 1e3) / 1e9 / hbm_peak
                                for k, v in kinds.items()},
           "traffic": None, "peak_source": peak_source}
    if (dom == "flip" and FLIP_TRAFFIC and abs(w.p - FLIP_TRAFFIC_P) < 1e-12 and abs(w.q - FLIP_TRAFFIC_P) < 1e-12):
        out["traffic"] = FLIP_TRAFFIC * qubits * S          # bytes per launch (one application)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    units = {"noise": qubits, "syndrome": qubits, "pflip": qubits // 3}   # edges, faces, sites
    issue_peak = 152 * 4 * sm_mhz * 1e6                  # warp instructions per second
    inst_known = abs(w.p - SWEEP_INST_P) < 1e-12 and abs(w.q - SWEEP_INST_P) < 1e-12
    if inst_known:
        # the cycle's bound: every kernel at the slower of its HBM and issue bounds
        hbm = hbm_peak * 1e9
        b_noise = max(SWEEP_BYTES["noise"] * qubits * S / hbm, SWEEP_INST["noise"] * units["noise"] * words / issue_peak)
        b_syn = max(SWEEP_BYTES["syndrome"] * qubits * S / hbm,
                    SWEEP_INST["syndrome"] * units["syndrome"] * words / issue_peak)
        b_flip = SWEEP_BYTES["flip"] * qubits * S / hbm
        b_pflip = (max((SWEEP_BYTES["pflip"] - PFLIP_APPLY_BYTES) * qubits * S / hbm,
                       SWEEP_INST["pflip"] * units["pflip"] * words / issue_peak) + PFLIP_APPLY_BYTES * qubits * S / hbm)
        bound_s = b_noise + b_syn + per_step["flip"] * b_flip + per_step["pflip"] * b_pflip
        out["cycle_bound_ms"] = 1e3 * bound_s
        out["cycle_roofline_frac"] = bound_s / (ms / 1e3 / steps)
        out["cycle_roofline"] = ("sum over the cycle's kernels of max(algorithmic bytes / HBM peak, warp "
                                 "instructions / issue peak), decode kernels only (the readout is extra)")
    if inst_known and SWEEP_INST.get(dom):
        peak = issue_peak / 1e9
        achieved = SWEEP_INST[dom] * units[dom] * words / t_app / 1e9
        out.update(bound="alu", achieved=achieved, peak=peak, unit="Ginst/s", frac=achieved / peak,
                   peak_derivation=f"152 SMs x 4 schedulers x 1 warp instruction/clock x {sm_mhz:.0f} MHz")
    else:
        alg = SWEEP_BYTES[dom] * qubits * S
        achieved = alg / t_app / 1e9
        out.update(bound="hbm", achieved=achieved, peak=hbm_peak, unit="GB/s", frac=achieved / hbm_peak,
                   algorithmic_bytes_per_application=alg)
    return out


def cuda_arm(args):
    import torch
    import torch.distributed as dist

    import paper_2212_06985_gb300 as t3d

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = inp.WORKLOADS[args.workload]
    S = args.samples or w.n_samples
    sample0 = t3d.replica_sample0(rank, S)
    sizes = w.sizes
    W = inp.words_for(S)
    kw = dict(use_bp=w.decoder.startswith("bp"), bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes,
              schedule=w.schedule, n_apply=w.n_apply)
    chunk = bp_chunk(max(sizes), S)
    cfg = t3d.make_run_cfg(w.L, 1, w.p, w.q, w.seed, S, sample0=sample0, bp_chunk_samples=chunk, **kw)
    stream = torch.cuda.Stream(device=dev)
    states = [torch.zeros((inp.n_bits(L), W), dtype=torch.int64, device=dev) for L in sizes]
    masks = [torch.zeros(S, dtype=torch.uint8, device=dev) for _ in sizes]
    counts = [torch.zeros(8, dtype=torch.int64, device=dev) for _ in sizes]
    batch = t3d.make_batch([dict(L=L, n_samples=S, sample0=sample0, e=e, mask=m, counts8=c)
                            for L, e, m, c in zip(sizes, states, masks, counts)])
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev)
    qubits = sum(inp.n_bits(L) for L in sizes)
    torch.cuda.synchronize()

    def step(t):
        cfg.cycle0 = t
        t3d.toric3d_run_batch(cfg, batch, work, stream=stream)

    tuned = None
    with torch.cuda.stream(stream):
        if kw["use_bp"] and not args.no_autotune:
            cap, ms_it = t3d.toric3d_autotune_batch(cfg, batch, work, stream=stream)
            tuned = {"bp_step_blocks_per_sm": cap, "bp_step_ms": ms_it}
        for t in range(args.warmup):
            step(t)
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    t3d.toric3d_profile_reset()
    t3d.toric3d_profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for t in range(args.warmup, args.warmup + args.steps):
            step(t)
        ev1.record(stream)
    ev1.synchronize()
    t3d.toric3d_profile_enable(False)
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = {k: t3d.toric3d_profile_read(k) for k in t3d.KERNEL_KINDS}
    t3d.toric3d_profile_reset()
    launches = sum(v[1] for v in prof.values())

    t_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms = float(t_max.item())
    total_qc = qubits * S * world * args.steps
    value = total_qc / (ms / 1e3)

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_source = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6.8 TB/s"
    if kw["use_bp"]:
        # dominant kernel: BP iteration (algorithmic bytes per edge-sample: 16 B read + 16 B
        # written; the first iteration of each chunk reads nothing)
        bp_ms, bp_launches = prof["bp_step"]
        rounds = math.ceil(S / chunk)
        alg_bytes = qubits * S * args.steps * (32.0 * (w.bp_iters - 1) + 16.0)
        achieved = alg_bytes / (bp_ms / 1e3) / 1e9 if bp_ms > 0 else 0.0
        traffic = None
        if BP_STEP_TRAFFIC and bp_launches:
            traffic = qubits * S * args.steps * (BP_STEP_TRAFFIC["first_iteration"] +
                                                 BP_STEP_TRAFFIC["full_iteration"] * (w.bp_iters - 1)) / bp_launches
        roofline = {"kernel": "k_bp_step", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": peak_source,
                    "launches": bp_launches, "avg_launch_ms": bp_ms / max(bp_launches, 1),
                    "share_of_step": bp_ms / ms if ms else None,
                    "expected_launches": w.bp_iters * rounds * args.steps,
                    "algorithmic_bytes_per_launch": alg_bytes / max(bp_launches, 1)}
    else:
        roofline = sweep_roofline(prof, w, qubits, S, args.steps, ms, hbm_peak, peak_source, clk)

    # end-to-end: every step uploads each error state from pinned host memory, decodes one
    # cycle through the C ABI and downloads the state, the masks and the counts.  The batch
    # runs as --e2e-parts parts (consecutive 64-sample-aligned sample ranges, the same samples
    # as one batch) decoded one after the other on the compute stream, each part with its own
    # copy stream, so a part's copies overlap the other parts' decoding.
    e2e = None
    if not args.e2e_steps:
        args.e2e_steps = max(3, args.steps)
    if not args.no_e2e:
        step_s = max(64, (S // max(1, args.e2e_parts) + 63) // 64 * 64)
        parts = [(off, min(step_s, S - off)) for off in range(0, S, step_s)]
        halves = []
        for off, n in parts:
            hw = inp.words_for(n)
            h_states = [torch.empty((inp.n_bits(L), hw), dtype=torch.int64, device=dev) for L in sizes]
            h_masks = [torch.zeros(n, dtype=torch.uint8, device=dev) for _ in sizes]
            h_counts = [torch.zeros(8, dtype=torch.int64, device=dev) for _ in sizes]
            h_host = [torch.empty((inp.n_bits(L), hw), dtype=torch.int64, pin_memory=True) for L in sizes]
            for hh, e in zip(h_host, states):
                hh.copy_(e[:, off // 64:off // 64 + hw])
            h_batch = t3d.make_batch([dict(L=L, n_samples=n, sample0=sample0 + off, e=e, mask=m, counts8=c)
                                      for L, e, m, c in zip(sizes, h_states, h_masks, h_counts)])
            h_cfg = t3d.make_run_cfg(w.L, 1, w.p, w.q, w.seed, n, sample0=sample0 + off,
                                     bp_chunk_samples=chunk, **kw)
            assert t3d.toric3d_run_batch_workspace_bytes(h_cfg, h_batch) <= work.numel()
            halves.append(dict(n=n, states=h_states, masks=h_masks, counts=h_counts, host=h_host, batch=h_batch,
                               cfg=h_cfg, mask_host=[torch.empty(n, dtype=torch.uint8, pin_memory=True) for _ in sizes],
                               counts_host=[torch.empty(8, dtype=torch.int64, pin_memory=True) for _ in sizes],
                               cs=torch.cuda.Stream(device=dev), up=torch.cuda.Event(), done=torch.cuda.Event()))

        def e2e_step(i):
            for h in halves:                         # uploads (after the half's previous download)
                with torch.cuda.stream(h["cs"]):
                    for d_e, h_e in zip(h["states"], h["host"]):
                        d_e.copy_(h_e, non_blocking=True)
                    h["up"].record(h["cs"])
            for h in halves:                         # decoding, one half after the other
                stream.wait_event(h["up"])
                h["cfg"].cycle0 = args.warmup + args.steps + i
                t3d.toric3d_run_batch(h["cfg"], h["batch"], work, stream=stream)
                h["done"].record(stream)
                with torch.cuda.stream(h["cs"]):     # downloads
                    h["cs"].wait_event(h["done"])
                    for d_e, h_e in zip(h["states"], h["host"]):
                        h_e.copy_(d_e, non_blocking=True)
                    for mh, m in zip(h["mask_host"], h["masks"]):
                        mh.copy_(m, non_blocking=True)
                    for ch, c in zip(h["counts_host"], h["counts"]):
                        ch.copy_(c, non_blocking=True)

        E2E_WARMUP = 2                               # untimed, like the device-timed steps' warm-up
        for i in range(E2E_WARMUP):
            e2e_step(i)
        for h in halves:
            h["cs"].synchronize()
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(E2E_WARMUP, E2E_WARMUP + args.e2e_steps):
            e2e_step(i)
        for h in halves:
            h["cs"].synchronize()
        stream.synchronize()
        dt = time.perf_counter() - t0
        dt_t = torch.tensor([dt], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(dt_t, op=dist.ReduceOp.MAX)
        dt = float(dt_t.item())
        state_bytes = sum(e.numel() * 8 for h in halves for e in h["states"])
        e2e = {"value": qubits * S * world * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes,
               "d2h_bytes_per_step": state_bytes + sum(h["n"] + 64 for h in halves) * len(sizes),
               "steps": args.e2e_steps, "ms_per_step": 1e3 * dt / args.e2e_steps,
               "warmup": 2,
               "note": "error states uploaded from and downloaded to pinned host memory every step, "
                       f"{len(parts)} parts whose copies overlap the other parts' decoding"}
        del halves

    fail_counts = [c.cpu().tolist() for c in counts]
    learned = None
    if not args.no_learned and w.decoder == "bp_pflip" and os.path.exists(WEIGHTS):
        del work
        learned = learned_leg(args, t3d, w, S, sample0, dev, stream, barrier, world, peaks)
        learned["vs_bp_pflip"] = learned["value"] / value
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(w, args.cpu_seconds)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "value_is": VALUE_IS, "unit": UNIT, "n_gpus": world,
                "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
                "data": "synthetic (seeded Philox phenomenological noise)",
                "config": dict(workload_config(w, S), parallelism=f"replicas{world}"),
                "samples_per_s": S * world * args.steps / (ms / 1e3) / 1,  # sample-cycles per second
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "kernels_ms": {k: v[0] for k, v in prof.items() if v[1]},
                "kernels_launches": {k: v[1] for k, v in prof.items() if v[1]},
                "clocks": clk, "autotune": tuned, "logical_counts": fail_counts,
                "logical_counts_after_cycles": args.warmup + args.steps,
                "learned_pflip": learned}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return cuda_arm(args)


if __name__ == "__main__":
    sys.exit(main())
