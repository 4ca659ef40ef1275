"""Threshold experiments of the paper, run with the library's whole-run call.

Presets (phenomenological noise, p = q, readout by majority vote on the
logical Z lines of the final error, no noiseless round):
  flip : one parallel flip application per code cycle, 1000 cycles (Sec. 3.1, Fig. 2)
  bp   : 30 BP iterations per cycle, 500 cycles (Sec. 4.1, Fig. 6)
  pbp  : 20 BP iterations then P F F P F F, 500 cycles (Sec. 4.2, Fig. 7)
  table1 --nA n --lp l : n rule applications per cycle, every l-th one p-flip,
         1000 cycles (Sec. 3.2, Table 1)
  --meta-checks : the BP presets with the cube meta-checks (Sec. 4.1, last
         paragraph; the paper proposes them without simulating them)
  table1-sweep : every non-empty cell of Table 1 on a 0.1% grid around the
         paper's value, L = 14 and 24; one line per cell with the crossing
  table2 : p-BP at L = 14, 500 cycles (App. A.2, Table 2), the histogram of
         the eight logical error patterns set against the paper's by a
         chi-square test of homogeneity (patterns pooled by weight, the code
         being symmetric under axis permutations), over all runs and over
         the failed runs alone
  --reading r : bp / pbp / table2 under another reading of BP inside a run
         (readings.py: restart, warm, halfiter, measdecide), composed from the
         library's single-step calls

  python -m paper_2212_06985_gb300.threshold pbp --L 14 18 24 32 --p 0.053 0.054 0.055 0.056 --samples 10000

Each (L, p) point prints one JSON line with the failure counts of logical
qubit 0 (the paper plots one of the three; the code is symmetric) and of
any qubit.  The last line gives the crossing read from the data (between the
last rate where the largest L fails less often than the smallest and the
next) and, with enough unsaturated points, the fit of the paper's ansatz
p_fail = a0 + a1 x + a2 x^2, x = (p - p_th) L^(1/nu) (Sec. 3.2, after Table 1).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import (make_batch, make_run_cfg, n_bits, table1_schedule, toric3d_run_batch,
               toric3d_run_batch_workspace_bytes, words_for)
from .readings import READINGS, run_stepwise

PRESETS = {
    "flip": dict(T=1000, use_bp=False, bp_iters=0, schedule="F", n_apply=1),
    "bp": dict(T=500, use_bp=True, bp_iters=30, schedule="", n_apply=0),
    "pbp": dict(T=500, use_bp=True, bp_iters=20, schedule="PFFPFF", n_apply=6),
    "table1": dict(T=1000, use_bp=False, bp_iters=0, schedule="", n_apply=0),   # schedule from (n_A, lambda_p)
}


def run_point(preset: str, L: int, p: float, samples: int, seed: int, T: int | None = None,
              meas_nodes: bool = True, n_A: int = 5, lambda_p: int = 3, meta_checks: bool = False,
              reading: str | None = None, device="cuda:0") -> dict:
    """One whole run of `samples` codes; returns failure counts and the run time.
    reading (bp / pbp only): compose the run step by step under that reading of
    BP inside a run (readings.py) instead of the whole-run call."""
    pr = dict(PRESETS[preset])
    if T is not None:
        pr["T"] = T
    if reading is not None:
        if not pr["use_bp"] or meta_checks or not meas_nodes:
            raise ValueError("--reading applies to the bp / pbp presets with measurement variables")
        r = run_stepwise(L, p, p, samples, seed, pr["T"], pr["bp_iters"], pr["schedule"], pr["n_apply"],
                         reading, device=device)
        r.update(preset=preset, meas_nodes=True, meta_checks=False)
        return r
    if preset == "table1":
        pr["schedule"], pr["n_apply"] = table1_schedule(n_A, lambda_p), n_A
    dev = torch.device(device)
    e = torch.zeros((n_bits(L), words_for(samples)), dtype=torch.int64, device=dev)
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    batch = make_batch([dict(L=L, n_samples=samples, e=e, counts8=counts)])
    cfg = make_run_cfg(L, pr["T"], p, p, seed, samples, use_bp=pr["use_bp"], bp_iters=pr["bp_iters"],
                       bp_meas_nodes=meas_nodes, bp_meta_checks=meta_checks, schedule=pr["schedule"],
                       n_apply=pr["n_apply"])
    work = torch.empty(toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    toric3d_run_batch(cfg, batch, work)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c = counts.cpu().numpy()
    fail0 = int(c[1::2].sum())          # mask values with bit 0 set
    return {"preset": preset, "schedule": pr["schedule"], "L": L, "p": p, "T": pr["T"], "meas_nodes": meas_nodes,
            "meta_checks": meta_checks,
            "samples": samples,
            "seed": seed,
            "fail_q0": fail0, "fail_any": int(c[1:].sum()), "counts8": c.tolist(), "seconds": dt}


# Table 1 of the paper: thresholds (%) of flip + p-flip after 1000 cycles, keyed by
# (n_A, lambda_p); lambda_p > n_A means n_A flip applications and no p-flip.
TABLE1_PAPER = {(9, 2): 4.343, (9, 3): 4.652, (9, 4): 4.753, (9, 5): 4.652, (9, 6): 4.654,
                (7, 2): 4.212, (7, 3): 4.629, (7, 4): 4.615, (7, 5): 4.620, (7, 6): 4.558,
                (5, 2): 3.998, (5, 3): 4.445, (5, 4): 4.475, (5, 5): 4.274, (5, 6): 4.082,
                (3, 2): 3.604, (3, 3): 3.752, (3, 4): 3.943, (1, 2): 2.611}


def table1_sweep(Ls=(14, 24), samples: int = 3000, seed: int = 7000):
    """Yield, for every cell of Table 1, the failure rates on the 0.1% grid from 0.2%
    below to 0.2% above the paper's value (rounded to 0.1%) and the crossing."""
    for (nA, lp), th in sorted(TABLE1_PAPER.items()):
        centre = round(th, 1)
        grid = [round((centre + 0.1 * k) / 100, 4) for k in range(-2, 3)]
        pts = [run_point("table1", L, p, samples, seed + 100 * nA + 10 * lp + k + L, n_A=nA, lambda_p=lp)
               for L in Ls for k, p in enumerate(grid)]
        c = crossing_guess(pts)
        yield {"nA": nA, "lp": lp, "paper_pct": th, "crossing_pct": None if c is None else round(100 * c, 3),
               "rates": {f"L{q['L']}@{q['p']}": q["fail_q0"] / q["samples"] for q in pts}}


# Table 2 of the paper (App. A.2): logical X error patterns over the three encoded
# qubits after 500 cycles of p-BP at L = 14, p = q = 5.44% (printed "0.544"), 1000 runs.
TABLE2_PAPER = {"000": 731, "100": 52, "010": 53, "001": 62, "110": 21, "101": 30, "011": 26, "111": 25}
TABLE2_SETUP = dict(L=14, p=0.0544, T=500, runs=1000)


def pattern_counts(counts8) -> dict:
    """Mask histogram (bit d = logical qubit d) -> {"abc": count}, a = qubit 0."""
    return {f"{m & 1}{(m >> 1) & 1}{(m >> 2) & 1}": int(counts8[m]) for m in range(8)}


def by_weight(patterns: dict) -> list[int]:
    """Pattern counts pooled by the number of failed logical qubits (0..3)."""
    w = [0, 0, 0, 0]
    for k, v in patterns.items():
        w[k.count("1")] += v
    return w


def table2_compare(counts8) -> dict:
    """Chi-square tests of homogeneity between a measured pattern histogram and
    Table 2, on the weight classes 0..3 (all runs) and 1..3 (failed runs only,
    the correlation structure whatever the overall failure rate)."""
    from scipy.stats import chi2_contingency
    ours = by_weight(pattern_counts(counts8))
    paper = by_weight(TABLE2_PAPER)
    out = {"weights": ours, "paper_weights": paper}
    for name, sl in (("all", slice(0, 4)), ("failed", slice(1, 4))):
        a, b = ours[sl], paper[sl]
        keep = [i for i in range(len(a)) if a[i] + b[i] > 0]
        if len(keep) < 2 or sum(a) == 0:
            out[name] = None
            continue
        chi2, pv, dof, _ = chi2_contingency([[a[i] for i in keep], [b[i] for i in keep]])
        out[name] = {"chi2": float(chi2), "dof": int(dof), "p_value": float(pv)}
    return out


def crossing_guess(points: list[dict]) -> float | None:
    """The rate where the largest lattice starts failing more often than the smallest:
    midpoint between the last p with f(L_max) < f(L_min) and the next p."""
    Ls = sorted({q["L"] for q in points})
    rate = {(q["L"], q["p"]): q["fail_q0"] / q["samples"] for q in points}
    ps = sorted({q["p"] for q in points if (Ls[0], q["p"]) in rate and (Ls[-1], q["p"]) in rate})
    for a, b in zip(ps, ps[1:]):
        if rate[(Ls[-1], a)] < rate[(Ls[0], a)] and rate[(Ls[-1], b)] >= rate[(Ls[0], b)]:
            return 0.5 * (a + b)
    return None


def fit_threshold(points: list[dict]) -> dict | None:
    """Least-squares fit of p_fail(q0) = a0 + a1 x + a2 x^2, x = (p - p_th) L^(1/nu), over the
    points that are neither empty nor saturated (0 < p_fail < 0.45); None when fewer than five
    such points or fewer than two sizes remain, {"error": ...} when the fit does not converge."""
    from scipy.optimize import curve_fit
    use = [q for q in points if 0 < q["fail_q0"] < 0.45 * q["samples"]]
    if len({q["L"] for q in use}) < 2 or len(use) < 5:
        return None
    L = np.array([q["L"] for q in use], dtype=float)
    p = np.array([q["p"] for q in use], dtype=float)
    f = np.array([q["fail_q0"] / q["samples"] for q in use])
    n = np.array([q["samples"] for q in use], dtype=float)
    sigma = np.sqrt(f * (1 - f) / n)

    def model(X, pth, nu, a0, a1, a2):
        x = (X[1] - pth) * X[0] ** (1.0 / nu)
        return a0 + a1 * x + a2 * x * x

    p0 = [crossing_guess(use) or float(np.median(p)), 1.0, float(np.median(f)), 1.0, 0.0]
    try:
        popt, pcov = curve_fit(model, np.vstack([L, p]), f, p0=p0, sigma=sigma, maxfev=20000)
    except (RuntimeError, ValueError) as exc:
        return {"error": str(exc), "points": len(use)}
    err = np.sqrt(np.diag(pcov))
    if not (np.isfinite(err[0]) and popt[1] > 0):
        return {"error": "fit did not determine p_th (transition too steep for the sampled rates)",
                "points": len(use)}
    return {"p_th": popt[0], "p_th_err": err[0], "nu": popt[1], "nu_err": err[1], "a": popt[2:].tolist(),
            "points": len(use)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("preset", choices=sorted(PRESETS) + ["table1-sweep", "table2"])
    ap.add_argument("--L", type=int, nargs="+", default=[14, 18, 24])
    ap.add_argument("--p", type=float, nargs="+", default=None, help="error rates (required but for table1-sweep)")
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--T", type=int, default=None, help="code cycles (default: the preset's)")
    ap.add_argument("--seed", type=int, default=2212)
    ap.add_argument("--nA", type=int, default=5, help="table1: rule applications per cycle")
    ap.add_argument("--lp", type=int, default=3, help="table1: every lp-th application is p-flip")
    ap.add_argument("--meta-checks", action="store_true",
                    help="BP with the cube meta-checks over the measurement variables (Sec. 4.1, last paragraph)")
    ap.add_argument("--no-meas-nodes", action="store_true",
                    help="BP without the measurement-error variables (checks taken as exact)")
    ap.add_argument("--reading", choices=READINGS, default=None,
                    help="bp / pbp / table2: compose the runs step by step under this reading of BP in a run")
    a = ap.parse_args(argv)
    if a.preset == "table2":
        ps = a.p or [TABLE2_SETUP["p"]]
        samples = a.samples if a.samples != 10000 else TABLE2_SETUP["runs"]
        for k, p in enumerate(ps):
            q = run_point("pbp", TABLE2_SETUP["L"] if a.L == [14, 18, 24] else a.L[0], p, samples,
                          a.seed + k, a.T, reading=a.reading)
            q["patterns"] = pattern_counts(q["counts8"])
            q["table2"] = table2_compare(q["counts8"])
            print(json.dumps(q), flush=True)
        return 0
    if a.preset == "table1-sweep":
        for row in table1_sweep(tuple(a.L) if a.L != [14, 18, 24] else (14, 24), a.samples, a.seed):
            print(json.dumps(row), flush=True)
        return 0
    if not a.p:
        ap.error("--p is required")
    points = []
    for L in a.L:
        for k, p in enumerate(a.p):
            q = run_point(a.preset, L, p, a.samples, a.seed + 1000 * L + k, a.T, not a.no_meas_nodes, a.nA, a.lp,
                          a.meta_checks, a.reading)
            points.append(q)
            print(json.dumps(q), flush=True)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        fit = fit_threshold(points)
    print(json.dumps({"crossing": crossing_guess(points), "fit": fit}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
