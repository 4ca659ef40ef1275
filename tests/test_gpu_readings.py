"""The BP readings of readings.py (Sec. 4.1 / 4.2 inside a multi-cycle run) on
the GPU: the step-by-step 'restart' run equals the library's whole-run call bit
for bit, and the 'warm' and 'measdecide' runs equal the same readings composed
from the oracle's BP (binary64) on small lattices, where no posterior of the
oracle lies within 1e-4 of the decision boundary."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
from paper_2212_06985_gb300 import readings
from gpu_util import dev, download_bits, workspace

pytestmark = pytest.mark.gpu


def oracle_run(reading, L, p, samples, seed, T, iters, schedule, n_apply):
    """The reading composed from the oracle's single steps; returns (e, min |l|)."""
    n = 3 * L ** 3
    e = np.zeros((samples, n), dtype=np.uint8)
    m = None
    margin = np.inf
    cptr, cvar = oracle.toric_tanner(L)
    for t in range(1, T + 1):
        e = oracle.noise_batch(L, e, p, seed, 0, t)
        s = oracle.measure_batch(L, e, p, seed, 0, t)
        if reading == "measdecide":
            # every face check also holds its measurement-error variable n + f
            cv = np.concatenate([cvar.reshape(n, 4), (n + np.arange(n))[:, None]], axis=1).reshape(-1)
            cp = 5 * np.arange(n + 1)
            prior = np.array([np.log((1 - p) / p)] * n + [np.log((1 - p) / p)] * n)
            e_ext = np.concatenate([e, np.zeros_like(e)], axis=1)
            e_ext, s, llr = oracle.tanner_bp_batch(cp, cv, e_ext, s, prior, iters)
            e = np.ascontiguousarray(e_ext[:, :n])
        else:
            m_in = m if reading == "warm" else None
            m, llr = oracle.bp_batch(L, s, p, p, True, iters, m_in=m_in)
            d = (llr < 0).astype(np.uint8)
            e ^= d
            s ^= oracle.syndrome_batch(L, d)
        margin = min(margin, float(np.abs(llr).min()))
        for k in range(n_apply):
            e, s = oracle.flip_batch(L, e, s, schedule[k % len(schedule)] == "P", seed, 0, t, k)
    return e, margin


@pytest.mark.parametrize("schedule,n_apply,iters", [("PFFPFF", 6, 6), ("", 0, 9)])
def test_restart_steps_equal_the_whole_run(schedule, n_apply, iters):
    L, S, T, p, seed = 6, 200, 5, 0.05, 31
    got = readings.run_stepwise(L, p, p, S, seed, T, iters, schedule, n_apply, "restart", return_state=True)
    cfg = t3d.make_run_cfg(L, T, p, p, seed, S, use_bp=True, bp_iters=iters, schedule=schedule, n_apply=n_apply)
    e = torch.zeros_like(got["e"])
    counts = torch.zeros(8, dtype=torch.int64, device=dev())
    t3d.toric3d_run_cycles(cfg, e, workspace(t3d.toric3d_run_workspace_bytes(cfg)), None, counts)
    torch.cuda.synchronize()
    assert torch.equal(e, got["e"])
    assert counts.cpu().tolist() == got["counts8"]


@pytest.mark.parametrize("reading", ["warm", "measdecide"])
def test_reading_matches_the_oracle(reading):
    L, S, T, p, seed, iters = 4, 128, 4, 0.05, 25, 5
    ora_e, margin = oracle_run(reading, L, p, S, seed, T, iters, "PFFPFF", 6)
    assert margin > 1e-4
    got = readings.run_stepwise(L, p, p, S, seed, T, iters, "PFFPFF", 6, reading, return_state=True)
    assert np.array_equal(download_bits(got["e"], S), ora_e)
    mask = oracle.logical_batch(L, ora_e)
    assert got["counts8"] == np.bincount(mask, minlength=8).tolist()


def test_warm_start_differs_from_restart():
    """The readings are different decoders: on a noisy run the kept messages change decisions."""
    L, S, T, p, seed, iters = 6, 512, 6, 0.06, 5, 4
    a = readings.run_stepwise(L, p, p, S, seed, T, iters, "", 0, "restart", return_state=True)
    b = readings.run_stepwise(L, p, p, S, seed, T, iters, "", 0, "warm", return_state=True)
    assert not torch.equal(a["e"], b["e"])
