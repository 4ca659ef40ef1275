"""Whole runs on the GPU against the oracle (bit-exact for flip and p-flip,
stepwise replay for BP + p-flip), plus the run-level invariants: CUDA-graph
replay equals direct launches, a run split at any cycle resumes exactly, and
disjoint sample ranges (the multi-GPU partition) reproduce one large batch."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu


def _gpu_run(cfg, e_bits=None):
    L, S = cfg.L, cfg.n_samples
    n = 3 * L ** 3
    e = upload_bits(e_bits) if e_bits is not None else torch.zeros((n, inp.words_for(S)),
                                                                    dtype=torch.int64, device=dev())
    work = workspace(t3d.toric3d_run_workspace_bytes(cfg))
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    counts = torch.zeros(8, dtype=torch.int64, device=dev())
    stream = torch.cuda.Stream() if cfg.use_graph else None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())   # inputs were written on the current stream
        with torch.cuda.stream(stream):
            t3d.toric3d_run_cycles(cfg, e, work, mask, counts)
        stream.synchronize()
    else:
        t3d.toric3d_run_cycles(cfg, e, work, mask, counts)
    torch.cuda.synchronize()
    return mask.cpu().numpy(), counts.cpu().numpy(), download_bits(e, S)


def _ocfg(w, **kw):
    base = dict(use_bp=w.decoder.startswith("bp"), bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes,
                schedule=w.schedule, n_apply=w.n_apply, perfect_round=w.perfect_round,
                perfect_max_sweeps=w.perfect_max_sweeps)
    base.update(kw)
    return base


def test_flip_L4_workload_bit_exact_on_all_samples():
    w = inp.WORKLOADS["flip_L4"]
    kw = _ocfg(w)
    cfg = t3d.make_run_cfg(w.L, w.T, w.p, w.q, w.seed, w.n_samples, **kw)
    mask, counts, e = _gpu_run(cfg)
    ora_mask, ora_e = oracle.run_batch(oracle.make_cfg(w.L, w.T, w.p, w.q, w.seed, **kw), 0, w.n_samples)
    assert np.array_equal(mask, ora_mask)
    assert np.array_equal(e, ora_e)
    assert np.array_equal(counts, np.bincount(ora_mask, minlength=8))


@pytest.mark.parametrize("L,p", [(8, 0.03), (12, 0.045), (16, 0.05)])
def test_pflip_runs_bit_exact_on_subsample(L, p):
    S = 4096
    kw = dict(schedule="FFPFF", n_apply=5)
    cfg = t3d.make_run_cfg(L, L, p, p, 1000 + L, S, **kw)
    mask, counts, e = _gpu_run(cfg)
    k = 128 if L < 16 else 64
    ora_mask, ora_e = oracle.run_batch(oracle.make_cfg(L, L, p, p, 1000 + L, **kw), 0, k)
    assert np.array_equal(mask[:k], ora_mask)
    assert np.array_equal(e[:k], ora_e)
    assert counts.sum() == S


def test_graph_replay_equals_direct_launches():
    kw = dict(schedule="PFFPFF", n_apply=12, use_bp=True, bp_iters=6)
    a = _gpu_run(t3d.make_run_cfg(6, 5, 0.04, 0.04, 2, 1000, **kw))
    b = _gpu_run(t3d.make_run_cfg(6, 5, 0.04, 0.04, 2, 1000, use_graph=True, **kw))
    c = _gpu_run(t3d.make_run_cfg(6, 5, 0.04, 0.04, 2, 1000, use_graph=True, **kw))  # cached exec
    for x, y in ((a, b), (a, c)):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))


@pytest.mark.parametrize("use_bp", [False, True])
def test_split_run_resumes_exactly(use_bp):
    kw = dict(schedule="PFFPFF", n_apply=6, use_bp=use_bp, bp_iters=5)
    L, S, seed = 5, 700, 4
    full = _gpu_run(t3d.make_run_cfg(L, 6, 0.04, 0.04, seed, S, **kw))
    _, _, e_half = _gpu_run(t3d.make_run_cfg(L, 3, 0.04, 0.04, seed, S, **kw))
    second = _gpu_run(t3d.make_run_cfg(L, 3, 0.04, 0.04, seed, S, cycle0=3, **kw), e_half)
    assert np.array_equal(full[0], second[0]) and np.array_equal(full[2], second[2])


def test_disjoint_sample_ranges_reproduce_one_batch():
    kw = dict(schedule="FFPFF", n_apply=5)
    L, seed = 6, 8
    whole = _gpu_run(t3d.make_run_cfg(L, 4, 0.04, 0.04, seed, 640, **kw))
    parts = [_gpu_run(t3d.make_run_cfg(L, 4, 0.04, 0.04, seed, 320, sample0=o, **kw)) for o in (0, 320)]
    assert np.array_equal(whole[0], np.concatenate([parts[0][0], parts[1][0]]))
    assert np.array_equal(whole[1], parts[0][1] + parts[1][1])


def test_bp_pflip_cycles_replay_against_oracle():
    """Stepwise replay of a BP + p-flip run: both sides advance from the same
    state each cycle; BP decisions must agree wherever |l| > 1e-4, and the rest
    of the cycle (noise, measurement, p-flip schedule) must be bit-exact."""
    L, S, p, iters, T, seed = 6, 256, 0.04, 16, 4, 21
    n = 3 * L ** 3
    e = torch.zeros((n, inp.words_for(S)), dtype=torch.int64, device=dev())
    s = torch.zeros_like(e)
    work = workspace(t3d.toric3d_bp_workspace_bytes(L, S))
    fwork = workspace(t3d.toric3d_flip_workspace_bytes(L, e.shape[1]))
    llr = torch.zeros((n, S), dtype=torch.float32, device=dev())
    ora_e = np.zeros((S, n), np.uint8)
    ambiguous = 0
    for t in range(1, T + 1):
        t3d.toric3d_noise(L, e, p, seed, 0, t)
        t3d.toric3d_syndrome(L, e, s, p, seed, 0, t)
        ora_e = oracle.noise_batch(L, ora_e, p, seed, 0, t)
        ora_s = oracle.measure_batch(L, ora_e, p, seed, 0, t)
        assert np.array_equal(download_bits(e, S), ora_e) and np.array_equal(download_bits(s, S), ora_s)
        t3d.toric3d_bp(L, S, e, s, p, p, iters, work, llr)
        g = llr.cpu().numpy().T.astype(np.float64)
        _, ref = oracle.bp_batch(L, ora_s, p, p, True, iters)
        clear = np.abs(ref) > 1e-4
        ambiguous += int((~clear).sum())
        assert np.array_equal((g < 0)[clear], (ref < 0)[clear])
        d = (g < 0).astype(np.uint8)        # replay: the oracle takes the GPU's decisions
        ora_e, ora_s = ora_e ^ d, ora_s ^ oracle.syndrome_batch(L, d)
        t3d.toric3d_pflip(L, e, s, "PFFPFF", 6, 0, seed, 0, t, fwork)
        for k in range(6):
            ora_e, ora_s = oracle.flip_batch(L, ora_e, ora_s, "PFFPFF"[k] == "P", seed, 0, t, k)
        assert np.array_equal(download_bits(e, S), ora_e) and np.array_equal(download_bits(s, S), ora_s)
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, S, e, mask)
    assert np.array_equal(mask.cpu().numpy(), oracle.logical_batch(L, ora_e))
    print(f"ambiguous BP lanes (|l| <= 1e-4): {ambiguous}")
