"""Training and evaluation of the learned local pre-decoder.

Host-side orchestration only: every step (noise, measurement, BP, flip and
p-flip, the network's forward and backward passes, Adam) runs in the library's
CUDA kernels through the C ABI.

Training pairs come from the simulator itself: ensembles of codes are run
cycle by cycle under phenomenological noise and decoded by BP + p-flip (the
teacher); at every cycle the two most recent measured syndromes
(s_{t-1}, s_t) and the error e_t present just before decoding form one batch,
and the network is trained to predict e_t (mean binary cross-entropy).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import (make_batch, make_run_cfg, n_bits, toric3d_bp, toric3d_bp_workspace_bytes, toric3d_cnn_decode,
               toric3d_run_batch, toric3d_run_batch_workspace_bytes,
               toric3d_cnn_param_count, toric3d_cnn_blob_bytes, toric3d_cnn_prepare,
               toric3d_cnn_train_step, toric3d_cnn_train_workspace_bytes, toric3d_cnn_workspace_bytes,
               toric3d_flip_workspace_bytes, toric3d_logical, toric3d_noise, toric3d_pflip,
               toric3d_syndrome, words_for)

C, IN_C = 16, 6
_SHAPES = [(C, IN_C, 3, 3, 3), (C,), (C, C, 3, 3, 3), (C,), (C, C, 3, 3, 3), (C,), (3, C), (3,)]


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, small biases (FP32, the ABI's PyTorch order)."""
    rng = np.random.default_rng(seed)
    out = []
    for shape in _SHAPES:
        n = int(np.prod(shape))
        if len(shape) > 1:
            out.append(rng.normal(0.0, math.sqrt(2.0 / int(np.prod(shape[1:]))), n))
        else:
            out.append(np.zeros(n))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == toric3d_cnn_param_count()
    return p


@dataclasses.dataclass
class Decoder:
    """Decoder settings shared by the teacher and the learned path."""

    p: float
    q: float
    seed: int
    bp_iters: int = 16
    schedule: str = "PFFPFF"
    n_apply: int = 32


class Ensemble:
    """S independent codes of size L advanced one code cycle at a time."""

    def __init__(self, L: int, n_samples: int, dec: Decoder, device, sample0: int = 0):
        self.L, self.S, self.dec, self.dev, self.sample0 = L, n_samples, dec, device, sample0
        n, W = n_bits(L), words_for(n_samples)
        z = lambda: torch.zeros((n, W), dtype=torch.int64, device=device)
        self.e, self.s, self.s_prev, self.s_raw = z(), z(), z(), z()
        self.flip_work = torch.empty(toric3d_flip_workspace_bytes(L, W), dtype=torch.uint8, device=device)
        self.bp_work = None
        self.cnn_work = None
        self.t = 0

    def measure(self):
        """Qubit noise and one noisy measurement of cycle t+1 (s_prev keeps the last raw syndrome)."""
        self.t += 1
        d = self.dec
        toric3d_noise(self.L, self.e, d.p, d.seed, self.sample0, self.t)
        toric3d_syndrome(self.L, self.e, self.s, d.q, d.seed, self.sample0, self.t)
        self.s_raw.copy_(self.s)

    def decode_bp_pflip(self):
        d = self.dec
        if self.bp_work is None:
            chunk = min(self.S, 25024)
            self.bp_work = torch.empty(toric3d_bp_workspace_bytes(self.L, chunk), dtype=torch.uint8,
                                       device=self.dev)
        toric3d_bp(self.L, self.S, self.e, self.s, d.p, d.q, d.bp_iters, self.bp_work)
        self.schedule()

    def decode_learned(self, blob):
        if self.cnn_work is None:
            self.cnn_work = torch.empty(toric3d_cnn_workspace_bytes(self.L, self.S), dtype=torch.uint8,
                                        device=self.dev)
        toric3d_cnn_decode(self.L, self.S, self.s_prev, self.s, self.e, blob, self.cnn_work)
        self.schedule()

    def schedule(self):
        d = self.dec
        toric3d_pflip(self.L, self.e, self.s, d.schedule, d.n_apply, 0, d.seed, self.sample0, self.t,
                      self.flip_work)

    def end_cycle(self):
        self.s_prev.copy_(self.s_raw)

    def logical(self):
        mask = torch.zeros(self.S, dtype=torch.uint8, device=self.dev)
        counts = torch.zeros(8, dtype=torch.int64, device=self.dev)
        toric3d_logical(self.L, self.S, self.e, mask, counts)
        return counts.cpu().numpy()


def lr_at(step: int, steps: int, lr: float, warmup: int = 100) -> float:
    """Linear warm-up, then cosine decay to 5% of lr."""
    if step <= warmup:
        return lr * step / warmup
    x = (step - warmup) / max(1, steps - warmup)
    return lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * x)))


def train(L: int = 12, p=0.04, steps: int = 400, batch: int = 2048, lr: float = 2e-3,
          cycles_per_episode: int = 12, seed: int = 1, device="cuda:0", log_every: int = 50,
          init: np.ndarray | None = None):
    """Online training on simulator pairs; returns (params, loss history).

    Every step draws one fresh cycle of `batch` codes (episodes of
    cycles_per_episode cycles decoded by the BP + p-flip teacher), so the
    network sees steps * batch (syndrome pair, error) examples, each once.
    p (= q) is one rate or a list of rates taken by successive episodes."""
    rates = list(p) if isinstance(p, (list, tuple)) else [p]
    dev = torch.device(device)
    params = torch.from_numpy(init if init is not None else init_params(seed)).to(dev)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    blob = torch.empty(toric3d_cnn_blob_bytes(), dtype=torch.uint8, device=dev)
    toric3d_cnn_prepare(params, blob)
    work = torch.empty(toric3d_cnn_train_workspace_bytes(L, batch), dtype=torch.uint8, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    history = []
    ens = None
    episode = 0
    acc = torch.zeros(1, dtype=torch.float64, device=dev)
    n_acc = 0
    for step in range(1, steps + 1):
        if ens is None or ens.t >= cycles_per_episode:
            episode += 1
            pe = rates[(episode - 1) % len(rates)]
            ens = Ensemble(L, batch, Decoder(pe, pe, seed * 1000003 + episode), dev)
            ens.measure()
            ens.decode_bp_pflip()
            ens.end_cycle()
        ens.measure()
        toric3d_cnn_train_step(L, batch, ens.s_prev, ens.s, ens.e, params, m, v, step, lr_at(step, steps, lr),
                               blob, work, loss)
        acc += loss
        n_acc += 1
        ens.decode_bp_pflip()
        ens.end_cycle()
        if step % log_every == 0 or step == steps:
            history.append((step, float(acc.item()) / (n_acc * 3 * L ** 3 * batch)))
            acc.zero_()
            n_acc = 0
    return params.cpu().numpy(), history


BP_CHUNK_BYTES = 48 << 30


def evaluate(L: int, p: float, T: int, n_samples: int, params: np.ndarray | None, seed: int,
             fallback_max_weight: int = -1, dec: Decoder | None = None, use_graph: bool = True,
             device="cuda:0", fallback_sigmas: float = 0.0):
    """One whole run of T noisy cycles through toric3d_run_batch, decoded by
    BP + p-flip (params is None) or by the learned pre-decoder + p-flip (with
    the BP + p-flip fallback when fallback_max_weight >= 0).  Returns the
    logical-outcome counts, the run's device time in ms and the number of
    64-sample words sent to the fallback."""
    dev = torch.device(device)
    dec = dec or Decoder(p, p, seed)
    n, W = n_bits(L), words_for(n_samples)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev)
    s_prev = torch.zeros_like(e)
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    fb = torch.zeros(1, dtype=torch.int64, device=dev)
    blob = None
    if params is not None:
        blob = torch.empty(toric3d_cnn_blob_bytes(), dtype=torch.uint8, device=dev)
        toric3d_cnn_prepare(torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(dev), blob)
    batch = make_batch([dict(L=L, n_samples=n_samples, e=e, counts8=counts, s_prev=s_prev, fallback_words=fb)])
    # BP messages of at most BP_CHUNK_BYTES at a time (all samples in one chunk would need
    # about 3 GB per 1000 samples at L = 32)
    per_word = toric3d_bp_workspace_bytes(L, 64)
    chunk = n_samples if W * per_word <= BP_CHUNK_BYTES else max(1, BP_CHUNK_BYTES // per_word) * 64
    cfg = make_run_cfg(L, T, p, dec.q, dec.seed, n_samples, use_bp=params is None, bp_iters=dec.bp_iters,
                       schedule=dec.schedule, n_apply=dec.n_apply, use_graph=use_graph, cnn_blob=blob,
                       fallback_max_weight=fallback_max_weight if params is not None else -1,
                       fallback_sigmas=fallback_sigmas if params is not None else 0.0,
                       bp_chunk_samples=chunk if params is None else 0)
    work = torch.empty(toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        toric3d_run_batch(cfg, batch, work)
        ev1.record(stream)
    stream.synchronize()
    return counts.cpu().numpy(), ev0.elapsed_time(ev1), int(fb.item())


def failure_rate(counts) -> float:
    """Fraction of samples with a logical error on any of the three logical qubits."""
    counts = np.asarray(counts)
    return float(counts[1:].sum() / max(1, counts.sum()))


def wilson_interval(k: int, n: int, z: float = 1.959964) -> tuple[float, float]:
    """95% Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return 0.0, 1.0
    ph = k / n
    den = 1 + z * z / n
    mid = (ph + z * z / (2 * n)) / den
    half = z * np.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / den
    return max(0.0, mid - half), min(1.0, mid + half)


def two_proportion_test(k1: int, n1: int, k2: int, n2: int) -> dict:
    """Is the second failure rate higher than the first?  One-sided pooled z-test and
    Fisher's exact test (the latter also where the counts are small or zero)."""
    from math import erf, sqrt
    p1, p2 = k1 / n1, k2 / n2
    pool = (k1 + k2) / (n1 + n2)
    se = sqrt(pool * (1 - pool) * (1 / n1 + 1 / n2))
    z = (p2 - p1) / se if se > 0 else 0.0
    out = {"z": z, "p_one_sided_z": 0.5 * (1 - erf(z / sqrt(2))) if se > 0 else 1.0}
    try:
        from scipy.stats import fisher_exact
        out["p_one_sided_fisher"] = float(fisher_exact([[k2, n2 - k2], [k1, n1 - k1]], alternative="greater")[1])
    except ImportError:
        pass
    return out


def save_params(path: str, params: np.ndarray, **meta):
    np.savez(path, params=np.asarray(params, dtype=np.float32),
             **{k: np.asarray(v) for k, v in meta.items()})


def load_params(path: str) -> np.ndarray:
    with np.load(path) as z:
        p = np.array(z["params"], dtype=np.float32)
    assert p.size == toric3d_cnn_param_count()
    return p


def _main(argv=None):
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description="train or evaluate the learned pre-decoder")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train", help="online training at L, p = q (BP + p-flip teacher)")
    t.add_argument("--L", type=int, default=12)
    t.add_argument("--p", type=float, nargs="+", default=[0.04], help="noise rate(s), one per episode in turn")
    t.add_argument("--steps", type=int, default=5000)
    t.add_argument("--batch", type=int, default=2048)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=1)
    t.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights", "cnn_L12_p04.npz"))
    e = sub.add_parser("evaluate", help="logical failures and time of BP + p-flip and learned + p-flip runs")
    e.add_argument("--L", type=int, default=24)
    e.add_argument("--p", type=float, nargs="+", default=[0.04])
    e.add_argument("--samples", type=int, default=100_000)
    e.add_argument("--T", type=int, default=0, help="cycles (default L)")
    e.add_argument("--seed", type=int, default=1234)
    e.add_argument("--fallback-max-weight", type=int, default=-1)
    e.add_argument("--fallback-sigmas", type=float, default=0.0,
                   help="add q 3L^3 + this many binomial standard deviations to the fallback threshold")
    e.add_argument("--weights", default=os.path.join(os.path.dirname(__file__), "weights", "cnn_L12_p04.npz"))
    e.add_argument("--no-bp", action="store_true", help="skip the BP + p-flip comparison run")
    a = ap.parse_args(argv)
    if a.cmd == "train":
        params, hist = train(L=a.L, p=a.p, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed,
                             log_every=max(1, a.steps // 25))
        save_params(a.out, params, steps=a.steps, batch=a.batch, L=a.L, p=np.asarray(a.p))
        print(json.dumps({"out": a.out, "loss": hist}))
        return 0
    params = load_params(a.weights)
    T = a.T or a.L
    for p in a.p:
        row = {"L": a.L, "p": p, "T": T, "samples": a.samples}
        legs = [("learned_pflip", params, a.fallback_max_weight)]
        if not a.no_bp:
            legs.insert(0, ("bp_pflip", None, -1))
        for name, prm, fb in legs:
            counts, ms, words = evaluate(a.L, p, T, a.samples, prm, a.seed, fallback_max_weight=fb,
                                         fallback_sigmas=a.fallback_sigmas)
            k = int(np.asarray(counts)[1:].sum())
            row[name] = {"failure_rate": failure_rate(counts), "failures": k,
                         "ci95": wilson_interval(k, a.samples), "counts": counts.tolist(), "ms": ms,
                         "qubit_cycles_per_s": n_bits(a.L) * a.samples * T / (ms / 1e3), "fallback_words": words,
                         "fallback_word_fraction": words / (T * words_for(a.samples))}
        if "bp_pflip" in row:
            row["learned_worse_than_bp"] = two_proportion_test(row["bp_pflip"]["failures"], a.samples,
                                                               row["learned_pflip"]["failures"], a.samples)
            row["speedup"] = row["learned_pflip"]["qubit_cycles_per_s"] / row["bp_pflip"]["qubit_cycles_per_s"]
        print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
