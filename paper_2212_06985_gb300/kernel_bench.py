"""Micro-benchmarks of single library calls on synthetic seeded inputs (for
profiling one kernel at a time; the whole-cycle benchmark is bench.py).

  python -m paper_2212_06985_gb300.kernel_bench cnn   --L 24 --samples 16384
  python -m paper_2212_06985_gb300.kernel_bench sweep --L 32 --samples 8192 --rule F
  python -m paper_2212_06985_gb300.kernel_bench cycle --L 32 --samples 8192 --schedule FFPFF
  python -m paper_2212_06985_gb300.kernel_bench bp    --L 32 --samples 1024
  python -m paper_2212_06985_gb300.kernel_bench bpmeta --L 24 --samples 1024
  python -m paper_2212_06985_gb300.kernel_bench tanner --n-classical 400 --samples 1024

The tanner case decodes the Z checks of the hypergraph product of two seeded
(3,4)-biregular classical codes (toric3d_inputs.hgp_workload; run from the
repository root): one p-flip application (PF, mean of the two) and BP.

Every line printed is one JSON object with the call's mean time over --reps
timed calls (CUDA events) after --warmup untimed ones.
"""
from __future__ import annotations

import argparse
import json
import os

import torch

from . import (n_bits, toric3d_bp, toric3d_bp_meta, toric3d_bp_meta_workspace_bytes, toric3d_bp_workspace_bytes, toric3d_cnn_blob_bytes, toric3d_cnn_decode,
               toric3d_cnn_prepare, toric3d_cnn_status, toric3d_cnn_workspace_bytes, toric3d_flip_workspace_bytes,
               toric3d_noise, toric3d_pflip, toric3d_syndrome, words_for)

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cnn_L12_p04.npz")
CNN_FLOP_PER_SITE = 2 * 27 * 16 * (6 + 16 + 16) + 2 * 16 * 3
# BP with meta-checks, FP32 messages, per qubit-sample and iteration: edge totals
# (read 4 face messages, write 1), faces (read 4 totals + 4 own messages + 2 cube
# messages, write 5), cubes (12 reads + 6 writes per cube, i.e. per 3 faces)
BP_META_BYTES = 4 * ((4 + 1) + (10 + 5) + (12 + 6) / 3)


def _timed(fn, warmup, reps):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def _state(L, S, p, seed, dev):
    """A code cycle's state: qubit noise and one noisy measurement at rate p."""
    e = torch.zeros((n_bits(L), words_for(S)), dtype=torch.int64, device=dev)
    s = torch.zeros_like(e)
    toric3d_noise(L, e, p, seed, 0, 1)
    toric3d_syndrome(L, e, s, p, seed, 0, 1)
    return e, s


def bench_cnn(a, dev):
    import numpy as np
    from .learned import load_params
    params = torch.from_numpy(load_params(a.weights) if os.path.exists(a.weights) else
                              np.zeros(16515, dtype=np.float32)).to(dev)
    blob = torch.empty(toric3d_cnn_blob_bytes(), dtype=torch.uint8, device=dev)
    toric3d_cnn_prepare(params, blob)
    e, s_prev = _state(a.L, a.samples, a.p, a.seed, dev)
    _, s = _state(a.L, a.samples, a.p, a.seed + 1, dev)
    work = torch.empty(toric3d_cnn_workspace_bytes(a.L, a.samples), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: toric3d_cnn_decode(a.L, a.samples, s_prev, s, e, blob, work), a.warmup, a.reps)
    toric3d_cnn_status()
    sites = a.L ** 3 * a.samples
    return {"call": "toric3d_cnn_decode", "L": a.L, "samples": a.samples, "ms": ms,
            "qubit_cycles_per_s": 3 * sites / (ms / 1e3),
            "algorithmic_tflops": CNN_FLOP_PER_SITE * sites / (ms / 1e3) / 1e12}


def bench_sweep(a, dev):
    e, s = _state(a.L, a.samples, a.p, a.seed, dev)
    W = words_for(a.samples)
    work = torch.empty(toric3d_flip_workspace_bytes(a.L, W), dtype=torch.uint8, device=dev)
    sched = a.rule * 2   # two applications per call (an even count leaves no copy-back)
    ms = _timed(lambda: toric3d_pflip(a.L, e, s, sched, 2, 0, a.seed, 0, 1, work), a.warmup, a.reps) / 2
    return {"call": "toric3d_pflip", "rule": a.rule, "L": a.L, "samples": a.samples, "ms_per_application": ms,
            "algorithmic_GBps": n_bits(a.L) * a.samples * 0.5 / (ms / 1e3) / 1e9}


def bench_cycle(a, dev):
    """One code cycle of the flip / p-flip decoders: qubit noise, the noisy
    measurement and the schedule (each call a new cycle index)."""
    W = words_for(a.samples)
    e = torch.zeros((n_bits(a.L), W), dtype=torch.int64, device=dev)
    s = torch.zeros_like(e)
    work = torch.empty(toric3d_flip_workspace_bytes(a.L, W), dtype=torch.uint8, device=dev)
    cyc = [0]

    def call():
        cyc[0] += 1
        toric3d_noise(a.L, e, a.p, a.seed, 0, cyc[0])
        toric3d_syndrome(a.L, e, s, a.p, a.seed, 0, cyc[0])
        toric3d_pflip(a.L, e, s, a.schedule, len(a.schedule), 0, a.seed, 0, cyc[0], work)

    ms = _timed(call, a.warmup, a.reps)
    return {"call": "noise + syndrome + toric3d_pflip", "schedule": a.schedule, "L": a.L, "samples": a.samples,
            "ms_per_cycle": ms, "qubit_cycles_per_s": n_bits(a.L) * a.samples / (ms / 1e3)}


def bench_bp(a, dev):
    e, s = _state(a.L, a.samples, a.p, a.seed, dev)
    work = torch.empty(toric3d_bp_workspace_bytes(a.L, a.samples), dtype=torch.uint8, device=dev)
    e0, s0 = e.clone(), s.clone()

    def call():
        e.copy_(e0)
        s.copy_(s0)
        toric3d_bp(a.L, a.samples, e, s, a.p, a.p, a.iters, work)

    ms = _timed(call, a.warmup, a.reps)
    return {"call": "toric3d_bp", "L": a.L, "samples": a.samples, "iters": a.iters, "ms": ms}


def bench_bp_meta(a, dev):
    e, s = _state(a.L, a.samples, a.p, a.seed, dev)
    work = torch.empty(toric3d_bp_meta_workspace_bytes(a.L, a.samples), dtype=torch.uint8, device=dev)
    e0, s0 = e.clone(), s.clone()

    def call():
        e.copy_(e0)
        s.copy_(s0)
        toric3d_bp_meta(a.L, a.samples, e, s, a.p, a.p, a.iters, work)

    ms = _timed(call, a.warmup, a.reps)
    qs = n_bits(a.L) * 64 * words_for(a.samples)
    return {"call": "toric3d_bp_meta", "L": a.L, "samples": a.samples, "iters": a.iters, "ms": ms,
            "algorithmic_GBps_iterations": BP_META_BYTES * qs * a.iters / (ms / 1e3) / 1e9}


def bench_tanner(a, dev):
    import toric3d_inputs
    from . import (tanner_prepare, toric3d_tanner_bp, toric3d_tanner_bp_workspace_bytes,
                   toric3d_tanner_flip_workspace_bytes, toric3d_tanner_noise, toric3d_tanner_pflip,
                   toric3d_tanner_syndrome)
    cptr, cvar, n = toric3d_inputs.hgp_workload(a.n_classical, a.seed)
    g = tanner_prepare(cptr, cvar, n, dev)
    S, W = a.samples, words_for(a.samples)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev)
    s = torch.zeros((g.n_checks, W), dtype=torch.int64, device=dev)
    toric3d_tanner_noise(g, S, e, a.p, a.seed, 0, 1)
    toric3d_tanner_syndrome(g, S, e, s, a.p, a.seed, 0, 1)
    fwork = torch.empty(toric3d_tanner_flip_workspace_bytes(g, S), dtype=torch.uint8, device=dev)
    ms_rule = _timed(lambda: toric3d_tanner_pflip(g, S, e, s, "PF", 2, 0, a.seed, 0, 1, fwork), a.warmup, a.reps) / 2
    prior = torch.full((n,), float(__import__("math").log((1 - a.p) / a.p)), dtype=torch.float32, device=dev)
    work = torch.empty(toric3d_tanner_bp_workspace_bytes(g, S), dtype=torch.uint8, device=dev)
    e0, s0 = e.clone(), s.clone()

    def bp():
        e.copy_(e0)
        s.copy_(s0)
        toric3d_tanner_bp(g, S, e, s, prior, a.iters, work)

    ms_bp = _timed(bp, a.warmup, a.reps)
    bp_bytes = (16 * g.n_edges + 4 * n) * 64 * W * a.iters   # FP32 messages, totals and gathers per iteration
    return {"call": "toric3d_tanner", "code": f"hgp({a.n_classical})", "n_vars": n, "n_checks": g.n_checks,
            "n_edges": g.n_edges, "samples": S, "ms_per_rule_application": ms_rule,
            "rule_variable_samples_per_s": n * 64 * W / (ms_rule / 1e3), "bp_iters": a.iters, "bp_ms": ms_bp,
            "bp_algorithmic_GBps": bp_bytes / (ms_bp / 1e3) / 1e9}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["cnn", "sweep", "cycle", "bp", "bpmeta", "tanner"])
    ap.add_argument("--schedule", default="FFPFF", help="cycle: the flip / p-flip schedule")
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--samples", type=int, default=16384)
    ap.add_argument("--p", type=float, default=0.04)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--rule", choices=["F", "P"], default="F")
    ap.add_argument("--iters", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--n-classical", type=int, default=400, help="tanner: bits of each classical code")
    a = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    out = {"cnn": bench_cnn, "sweep": bench_sweep, "cycle": bench_cycle, "bp": bench_bp, "bpmeta": bench_bp_meta, "tanner": bench_tanner}[a.what](a, dev)
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
