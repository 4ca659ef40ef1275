"""Readings of the paper's BP decoder inside a multi-cycle run (Sec. 4.1, 4.2).

Eqs. 1-4 fix one BP decode of one syndrome.  How BP sits inside a run of many
noisy code cycles is left open by the text; the whole-run call of the library
(``toric3d_run_batch``) takes one reading, and this module composes whole runs
from the library's single-step calls under the others the text allows, so
their thresholds can be set beside the paper's:

  restart     the library's reading: every cycle's BP starts from the priors
              (Eq. 1), the measurement-error variables enter as the constant
              factor tanh(l_q/2) of Eq. 2, and only qubits are corrected
              (l < 0).  Composed step by step it equals the whole-run call.
  warm        the check->variable messages of a cycle's last iteration start
              the next cycle's BP: the text initialises the messages from the
              priors and never says they are reset between cycles.
  halfiter    an "iteration" counted as one half-update (a factor update or a
              variable update), so the paper's 30 / 20 iterations are 15 / 10
              full ones.
  measdecide  the measurement-error variables are bits of the factor graph
              too, and the decoder corrects every bit whose posterior is below
              zero: a measurement variable below zero flips its syndrome bit
              before the flip / p-flip schedule runs.  (BP alone re-measures
              the next cycle, so this reading changes p-BP only.)

Every step runs in the library's kernels; this module only sequences calls.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import (n_bits, tanner_prepare, toric3d_bp_decide, toric3d_bp_decide_workspace_bytes,
               toric3d_bp_message_bytes, toric3d_bp_step, toric3d_flip_workspace_bytes, toric3d_logical,
               toric3d_noise, toric3d_pflip, toric3d_syndrome, toric3d_tanner_bp,
               toric3d_tanner_bp_workspace_bytes, words_for)

READINGS = ("restart", "warm", "halfiter", "measdecide")


def face_edges(L: int) -> np.ndarray:
    """int32 [3L^3][4]: the four edges of every face (Sec. 2), in the library's
    order: the face with normal n at r is spanned by the axes a < b other than
    n and holds the a-edges at r and r + e_b, then the b-edges at r and r + e_a."""
    f = np.arange(3 * L ** 3)
    n, x, y, z = f // L ** 3, f % L, (f // L) % L, (f // (L * L)) % L
    r = np.stack([x, y, z])
    out = np.empty((len(f), 4), dtype=np.int64)
    axes = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
    for nn, (a, b) in axes.items():
        sel = n == nn
        ra = r[:, sel]

        def edge(d, shift_axis):
            q = ra.copy()
            if shift_axis is not None:
                q[shift_axis] = (q[shift_axis] + 1) % L
            return ((d * L + q[2]) * L + q[1]) * L + q[0]

        out[sel, 0] = edge(a, None)
        out[sel, 1] = edge(a, b)
        out[sel, 2] = edge(b, None)
        out[sel, 3] = edge(b, a)
    return out.astype(np.int32)


def measurement_graph(L: int):
    """CSR of the face checks with one measurement-error variable each (Sec. 4.1):
    variables 0..n-1 are the qubits, n + f the measurement error of face f;
    check f acts on its four edges and on n + f."""
    n = n_bits(L)
    fe = face_edges(L)
    cvar = np.concatenate([fe, (n + np.arange(n, dtype=np.int32))[:, None]], axis=1).reshape(-1)
    cptr = (5 * np.arange(n + 1)).astype(np.int32)
    return cptr, cvar.astype(np.int32)


def prior_llr(p: float) -> float:
    return math.log((1.0 - p) / p)


def run_stepwise(L: int, p: float, q: float, samples: int, seed: int, T: int, bp_iters: int, schedule: str,
                 n_apply: int, reading: str = "restart", device="cuda:0", return_state: bool = False) -> dict:
    """A whole run (e = 0 at the start, cycles 1..T of noise, noisy measurement,
    BP under `reading`, then n_apply applications cycling through `schedule`;
    logical readout of the final error).  Returns the 8-pattern counts, and with
    return_state the final error words as "e" (int64 [3L^3][words], device)."""
    if reading not in READINGS:
        raise ValueError(f"reading must be one of {READINGS}")
    if not (0.0 < p < 0.5 and 0.0 < q < 0.5):
        raise ValueError("the BP readings need 0 < p, q < 1/2 (measurement variables on)")
    dev = torch.device(device)
    n, W = n_bits(L), words_for(samples)
    iters = bp_iters // 2 if reading == "halfiter" else bp_iters
    i64 = torch.int64
    if reading == "measdecide":
        # qubits and measurement variables share one state array; rows n.. hold the
        # measurement variables' (discarded) corrections
        e_ext = torch.zeros((2 * n, W), dtype=i64, device=dev)
        e = e_ext[:n]
        g = tanner_prepare(*measurement_graph(L), 2 * n, device=dev)
        prior = torch.tensor([prior_llr(p)] * n + [prior_llr(q)] * n, dtype=torch.float32, device=dev)
        bp_work = torch.empty(toric3d_tanner_bp_workspace_bytes(g, samples), dtype=torch.uint8, device=dev)
    else:
        e = torch.zeros((n, W), dtype=i64, device=dev)
        mb = toric3d_bp_message_bytes(L, samples)
        bufs = [torch.empty(mb // 4, dtype=torch.float32, device=dev) for _ in range(2)]
        dwork = torch.empty(toric3d_bp_decide_workspace_bytes(L, samples), dtype=torch.uint8, device=dev)
    s = torch.empty((n, W), dtype=i64, device=dev)
    fwork = torch.empty(toric3d_flip_workspace_bytes(L, W), dtype=torch.uint8, device=dev)
    counts = torch.zeros(8, dtype=i64, device=dev)
    cur = None
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for t in range(1, T + 1):
        toric3d_noise(L, e, p, seed, 0, t)
        toric3d_syndrome(L, e, s, q, seed, 0, t)
        if reading == "measdecide":
            toric3d_tanner_bp(g, samples, e_ext, s, prior, iters, bp_work)
        else:
            if reading != "warm":
                cur = None
            for _ in range(iters):
                out = bufs[1] if cur is bufs[0] else bufs[0]
                toric3d_bp_step(L, samples, s, p, q, cur, out)
                cur = out
            toric3d_bp_decide(L, samples, cur, p, e, s, dwork)
        if n_apply > 0:
            toric3d_pflip(L, e, s, schedule, n_apply, 0, seed, 0, t, fwork)
    toric3d_logical(L, samples, e, None, counts)
    torch.cuda.synchronize(dev)
    c = counts.cpu().numpy()
    out = {"reading": reading, "L": L, "p": p, "q": q, "T": T, "bp_iters": iters, "schedule": schedule,
           "samples": samples, "seed": seed, "fail_q0": int(c[1::2].sum()), "fail_any": int(c[1:].sum()),
           "counts8": c.tolist(), "seconds": time.perf_counter() - t0}
    if return_state:
        out["e"] = e.clone()
    return out
