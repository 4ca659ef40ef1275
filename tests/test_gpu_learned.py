"""Runs decoded by the learned pre-decoder (its convolution kernels are checked
against the PyTorch reference in test_gpu_cnn.py): the fallback gate against
syndrome weights counted on the CPU, and whole runs through
toric3d_run_batch against the same cycle assembled from the single-step entry
points (noise, measurement, pre-decoder, p-flip schedule, gate, and for the
flagged words only BP + schedule from the cycle's start, whose result replaces
the learned one)."""
import numpy as np
import pytest
import torch

import cnn_reference as ref
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,S", [(4, 200), (6, 64 * 40 + 5)])
def test_gate_matches_cpu_weights(L, S):
    n = 3 * L ** 3
    rng = np.random.default_rng(L)
    dens = rng.uniform(0.0, 0.3, S)
    bits = (rng.random((S, n)) < dens[:, None]).astype(np.uint8)
    s = upload_bits(bits)
    W = s.shape[1]
    weight = bits.sum(axis=1)
    work = workspace(t3d.toric3d_gate_workspace_bytes(L, W))
    for max_w in [0, int(np.median(weight)), int(weight.max()) - 1, int(weight.max()), 2 ** 31]:
        gate = torch.full((W,), 7, dtype=torch.uint8, device=dev())
        count = torch.zeros(1, dtype=torch.int64, device=dev())
        t3d.toric3d_gate(L, s, max_w, gate, work, count)
        torch.cuda.synchronize()
        pad = np.zeros(W * 64, dtype=np.int64)
        pad[:S] = weight
        want = (pad.reshape(W, 64) > max_w).any(axis=1)
        assert np.array_equal(gate.cpu().numpy().astype(bool), want), max_w
        assert int(count.item()) == int(want.sum())


def _blob(seed):
    blob = workspace(t3d.toric3d_cnn_blob_bytes())
    t3d.toric3d_cnn_prepare(torch.from_numpy(ref.random_params(seed)).to(dev()), blob)
    return blob


DEC = dict(p=0.04, seed=9, schedule="PFFPFF", n_apply=6, bp_iters=6)


def _stepwise(L, S, T, blob, max_w, sample0=0):
    """The learned cycle assembled from single-step calls."""
    n, W = 3 * L ** 3, inp.words_for(S)
    z = lambda: torch.zeros((n, W), dtype=torch.int64, device=dev())
    e, s, s_prev = z(), z(), z()
    flip_work = workspace(t3d.toric3d_flip_workspace_bytes(L, W))
    cnn_work = workspace(t3d.toric3d_cnn_workspace_bytes(L, S))
    bp_work = workspace(t3d.toric3d_bp_workspace_bytes(L, 64))
    w1_work = workspace(t3d.toric3d_flip_workspace_bytes(L, 1))
    p, seed = DEC["p"], DEC["seed"]
    flagged = 0
    for t in range(1, T + 1):
        t3d.toric3d_noise(L, e, p, seed, sample0, t)
        t3d.toric3d_syndrome(L, e, s, p, seed, sample0, t)
        s_raw = s.clone()
        e_pre = e.clone()
        t3d.toric3d_cnn_decode(L, S, s_prev, s, e, blob, cnn_work)
        t3d.toric3d_pflip(L, e, s, DEC["schedule"], DEC["n_apply"], 0, seed, sample0, t, flip_work)
        if max_w >= 0:
            weight = s.cpu().numpy().view(np.uint64)
            lanes = np.unpackbits(weight.view(np.uint8).reshape(n, W, 8), axis=2, bitorder="little")
            per_lane = lanes.sum(axis=0)                       # [W][64]
            for w in np.nonzero((per_lane > max_w).any(axis=1))[0]:
                flagged += 1              # decoded again from the cycle's start by BP + the schedule
                ew, sw = e_pre[:, w:w + 1].contiguous(), s_raw[:, w:w + 1].contiguous()
                t3d.toric3d_bp(L, 64, ew, sw, p, p, DEC["bp_iters"], bp_work)
                t3d.toric3d_pflip(L, ew, sw, DEC["schedule"], DEC["n_apply"], 0, seed, sample0 + 64 * int(w), t,
                                  w1_work)
                e[:, w:w + 1] = ew
                s[:, w:w + 1] = sw
        s_prev.copy_(s_raw)
    torch.cuda.synchronize()
    t3d.toric3d_cnn_status()
    return download_bits(e, S), download_bits(s_prev, S), flagged


def _run(L, S, T, blob, max_w, chunk=0, use_graph=False, split=None, sigmas=0.0):
    n, W = 3 * L ** 3, inp.words_for(S)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s_prev = torch.zeros_like(e)
    fb = torch.zeros(1, dtype=torch.int64, device=dev())
    counts = torch.zeros(8, dtype=torch.int64, device=dev())
    batch = t3d.make_batch([dict(L=L, n_samples=S, e=e, s_prev=s_prev, fallback_words=fb, counts8=counts)])
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())   # inputs were written on the current stream
    parts = [(0, T)] if split is None else [(0, split), (split, T - split)]
    with torch.cuda.stream(stream):
        for cycle0, t in parts:
            cfg = t3d.make_run_cfg(L, t, DEC["p"], DEC["p"], DEC["seed"], S, schedule=DEC["schedule"],
                                   n_apply=DEC["n_apply"], bp_iters=DEC["bp_iters"], cnn_blob=blob,
                                   fallback_max_weight=max_w, bp_chunk_samples=chunk, cycle0=cycle0,
                                   use_graph=use_graph, fallback_sigmas=sigmas)
            work = workspace(t3d.toric3d_run_batch_workspace_bytes(cfg, batch))
            t3d.toric3d_run_batch(cfg, batch, work)
    stream.synchronize()
    t3d.toric3d_cnn_status()
    return download_bits(e, S), download_bits(s_prev, S), int(fb.item()), counts.cpu().numpy()


@pytest.mark.parametrize("max_w,chunk", [(-1, 0), (0, 0), (60, 0), (10 ** 6, 0), (-1, 64), (60, 128)])
def test_learned_run_equals_stepwise(max_w, chunk):
    """chunk > 0 splits the samples into chunks that alternate between two streams."""
    L, S, T = 5, 200, 3
    blob = _blob(3)
    e_ref, sp_ref, flagged = _stepwise(L, S, T, blob, max_w)
    e, sp, fb, counts = _run(L, S, T, blob, max_w, chunk=chunk)
    print(f"max_weight {max_w}: {flagged} fallback words over {T} cycles")
    assert np.array_equal(e, e_ref)
    assert np.array_equal(sp, sp_ref)
    assert fb == flagged
    assert counts.sum() == S


def test_learned_run_chunks_graphs_and_splits_are_invisible():
    L, S, T = 4, 64 * 5 + 17, 4
    blob = _blob(5)
    base = _run(L, S, T, blob, 30)
    for kw in [dict(chunk=64), dict(chunk=128, use_graph=True), dict(split=1), dict(split=3, use_graph=True)]:
        got = _run(L, S, T, blob, 30, **kw)
        assert np.array_equal(got[0], base[0]), kw
        assert np.array_equal(got[1], base[1]), kw
        assert got[2] == base[2], kw
        assert np.array_equal(got[3], base[3]), kw


@pytest.mark.parametrize("L,S,sigmas", [(5, 200, 1.0), (4, 64 * 7 + 3, 0.5)])
def test_fallback_threshold_from_measurement_noise(L, S, sigmas):
    """fallback_sigmas adds floor(q n + k sqrt(q (1 - q) n)), n = 3L^3, to the threshold:
    the run equals the stepwise cycle gated at that weight, words past the first flagged
    ones included (the flagged words are compacted before BP and the schedule)."""
    n = 3 * L ** 3
    q = DEC["p"]
    thr = int(np.floor(q * n + sigmas * np.sqrt(q * (1 - q) * n)))
    blob = _blob(11)
    e_ref, sp_ref, flagged = _stepwise(L, S, 3, blob, thr)
    e, sp, fb, _ = _run(L, S, 3, blob, 0, sigmas=sigmas)
    print(f"threshold {thr}: {flagged} fallback words")
    assert flagged > 0
    assert np.array_equal(e, e_ref) and np.array_equal(sp, sp_ref) and fb == flagged
