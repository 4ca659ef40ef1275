"""The benchmark's other configurations at their full sizes, as whole runs through
the C ABI in the launch configuration the benchmark uses: p-flip at L = 16 with
10^6 samples, the benchmark's flip / p-flip workload (L = 32, 10^5 samples,
FFPFF), L = 16 and L = 24 mixed in one batch with BP16 + 32 x PFFPFF (10^5
samples each), and L = 48 with BP16 + 32 x PFFPFF (10^5 samples, BP in
chunks).  Whole batches are checked by properties that hold at any size (the
readout histogram, a batch equal to separate runs); sampled samples are
recomputed one by one by the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev
from oracle_pool import run_range, run_sample_if_clear, spawn_pool

pytestmark = pytest.mark.gpu


def _word_bits(words: torch.Tensor, w: int) -> np.ndarray:
    """[64][n] bits of the 64 samples of word w of a bit-sliced [n][W] tensor."""
    col = words[:, w].cpu().numpy().view(np.uint64)
    return ((col[None, :] >> np.arange(64, dtype=np.uint64)[:, None]) & np.uint64(1)).astype(np.uint8)


def _sample_bits(words: torch.Tensor, i: int) -> np.ndarray:
    return _word_bits(words, i // 64)[i % 64]


def _alloc(L, S):
    return (torch.zeros((inp.n_bits(L), inp.words_for(S)), dtype=torch.int64, device=dev()),
            torch.zeros(S, dtype=torch.uint8, device=dev()),
            torch.zeros(8, dtype=torch.int64, device=dev()))


def _check_readout(mask, counts, S):
    m, c = mask.cpu().numpy(), counts.cpu().numpy()
    assert c.sum() == S
    assert np.array_equal(np.bincount(m, minlength=8), c)
    return m


def _bp_oracle_lanes(L, w, kw, e, m, S, candidates, need):
    """Sampled samples of a one-cycle BP + p-flip run against the oracle (in a spawn pool),
    skipping a sample when one of its first-cycle posteriors lies within FP32 reach of zero
    (1e-4).  Only samples below n_samples: BP writes its decisions for a chunk's samples only,
    so the padding lanes of the last word are not decoded as the oracle decodes a sample."""
    assert all(i < S for i in candidates)
    with spawn_pool() as pool:
        results = pool.map(run_sample_if_clear, [(L, w.p, w.q, w.seed, i, w.bp_iters, kw) for i in candidates])
    checked = 0
    for r in results:
        if r is None:
            continue
        i, ora_e, ora_m = r
        assert np.array_equal(_sample_bits(e, i), ora_e), i
        assert m[i] == ora_m, i
        checked += 1
    assert checked >= need


def test_pflip_L16_million_samples():
    w = inp.WORKLOADS["pflip_L16"]
    L, S = w.L, w.n_samples
    kw = dict(schedule=w.schedule, n_apply=w.n_apply)
    cfg = t3d.make_run_cfg(L, w.T, w.p, w.q, w.seed, S, **kw)
    e, mask, counts = _alloc(L, S)
    work = torch.empty(t3d.toric3d_run_workspace_bytes(cfg), dtype=torch.uint8, device=dev())
    t3d.toric3d_run_cycles(cfg, e, work, mask, counts)
    torch.cuda.synchronize()
    m = _check_readout(mask, counts, S)
    ocfg = oracle.make_cfg(L, w.T, w.p, w.q, w.seed, **kw)
    W = inp.words_for(S)
    for wd in (0, W // 2, W - 1):          # the first, a middle and the last word, all 64 lanes
        ora_mask, ora_e = oracle.run_batch(ocfg, 64 * wd, 64)
        assert np.array_equal(_word_bits(e, wd), ora_e), wd
        assert np.array_equal(m[64 * wd:64 * wd + 64], ora_mask), wd
    del e, work
    torch.cuda.empty_cache()


def test_pflip_L32_full_size_as_the_bench_runs_it():
    """The flip / p-flip workload (L = 32, 10^5 samples, FFPFF) through toric3d_run_batch one
    cycle per call, as the benchmark times it (1024-thread flip tiles), three cycles; the first,
    a middle and the last (half-full) word against the oracle, one sample at a time."""
    w = inp.WORKLOADS["pflip_L32"]
    L, S, cycles = w.L, w.n_samples, 3
    kw = dict(schedule=w.schedule, n_apply=w.n_apply)
    e, mask, counts = _alloc(L, S)
    batch = t3d.make_batch([dict(L=L, n_samples=S, e=e, mask=mask, counts8=counts)])
    cfg = t3d.make_run_cfg(L, 1, w.p, w.q, w.seed, S, **kw)
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev())
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for t in range(cycles):
            cfg.cycle0 = t
            t3d.toric3d_run_batch(cfg, batch, work, stream=stream)
    stream.synchronize()
    del work
    m = _check_readout(mask, counts, S)
    W = inp.words_for(S)
    lanes = sorted(set(range(64)) | set(range(64 * (W // 2), 64 * (W // 2) + 64)) | set(range(64 * (W - 1), S)))
    with spawn_pool() as pool:
        got = pool.map(run_range, [(L, cycles, w.p, w.q, w.seed, kw, i, 1) for i in lanes])
    for i, (s0, ora_mask, ora_e) in zip(lanes, got):
        assert s0 == i
        assert np.array_equal(_sample_bits(e, i), ora_e[0]), i
        assert m[i] == ora_mask[0], i
    del e
    torch.cuda.empty_cache()


def test_mixed_L16_L24_batch_full_size():
    w = inp.WORKLOADS["bp_pflip_L16_L24"]
    S = w.n_samples
    kw = dict(use_bp=True, bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes, schedule=w.schedule,
              n_apply=w.n_apply)
    bufs = {L: _alloc(L, S) for L in w.sizes}
    batch = t3d.make_batch([dict(L=L, n_samples=S, e=bufs[L][0], mask=bufs[L][1], counts8=bufs[L][2])
                            for L in w.sizes])
    cfg = t3d.make_run_cfg(w.L, 1, w.p, w.q, w.seed, S, **kw)
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev())
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        t3d.toric3d_run_batch(cfg, batch, work, stream=stream)
    stream.synchronize()
    del work
    for L in w.sizes:
        # each item ends exactly where a run of that lattice alone ends
        e1, mask1, counts1 = _alloc(L, S)
        cfg1 = t3d.make_run_cfg(L, 1, w.p, w.q, w.seed, S, **kw)
        work1 = torch.empty(t3d.toric3d_run_workspace_bytes(cfg1), dtype=torch.uint8, device=dev())
        t3d.toric3d_run_cycles(cfg1, e1, work1, mask1, counts1)
        torch.cuda.synchronize()
        e, mask, counts = bufs[L]
        assert torch.equal(e, e1), L
        assert torch.equal(mask, mask1) and torch.equal(counts, counts1), L
        m = _check_readout(mask, counts, S)
        del e1, work1
        torch.cuda.empty_cache()
        _bp_oracle_lanes(L, w, kw, e, m, S, (0, 1, 63, 64, 25_000, 50_001, 77_777, 99_903, S - 2, S - 1), 4)


def test_bp_pflip_L48_full_size_sampled():
    w = inp.WORKLOADS["bp_pflip_L48"]
    L, S = w.L, w.n_samples
    kw = dict(use_bp=True, bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes, schedule=w.schedule,
              n_apply=w.n_apply)
    e, mask, counts = _alloc(L, S)
    cfg = t3d.make_run_cfg(L, 1, w.p, w.q, w.seed, S, bp_chunk_samples=8192, **kw)
    batch = t3d.make_batch([dict(L=L, n_samples=S, e=e, mask=mask, counts8=counts)])
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev())
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        t3d.toric3d_run_batch(cfg, batch, work, stream=stream)
    stream.synchronize()
    del work
    torch.cuda.empty_cache()
    m = _check_readout(mask, counts, S)
    # samples at the BP chunk boundaries (8192 samples), between them and at the batch's ends;
    # with 331,776 posteriors about nine in ten samples have one within 1e-4 of zero, hence
    # many candidates
    cands = sorted({0, 1, 63, 64, S - 2, S - 1} | {b + d for b in range(8192, S, 8192) for d in (-1, 0)} |
                   set(range(517, S, 1531)))
    _bp_oracle_lanes(L, w, kw, e, m, S, cands, 4)
    del e
    torch.cuda.empty_cache()
