"""The throughput workload at full size, in the launch configuration the
benchmark times: L = 32, p = q = 4%, 10^5 samples, one code cycle of BP16 +
32 x PFFPFF through toric3d_run_batch (BP in chunks of 25,024 samples, after
the BP autotuner has run).  Sampled samples are recomputed one by one by the
oracle; the whole batch is checked by properties that hold at any size.

BP at that size is also checked message by message (one whole 25,024-sample
chunk, 391 words, per-iteration protocol on three words across it) and over
four cycles of the benchmark's decoder, replayed lane by lane against the
oracle on lanes at the chunk boundaries."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, gpu_messages_to_oracle, message_index
from oracle_pool import bp_llr, bp_messages, spawn_pool
from test_gpu_bp import _input_rounding_bound, _tol

pytestmark = pytest.mark.gpu


def _sample_bits(words: torch.Tensor, i: int) -> np.ndarray:
    """Bits of sample i of a bit-sliced [n][W] tensor (one word column downloaded)."""
    col = words[:, i // 64].cpu().numpy().view(np.uint64)
    return ((col >> np.uint64(i % 64)) & np.uint64(1)).astype(np.uint8)


def test_bp_pflip_L32_full_size_sampled():
    w = inp.WORKLOADS["bp_pflip_L32"]
    L, S = w.L, w.n_samples
    n, W = inp.n_bits(L), inp.words_for(S)
    kw = dict(use_bp=True, bp_iters=w.bp_iters, bp_meas_nodes=w.bp_meas_nodes, schedule=w.schedule,
              n_apply=w.n_apply)
    cfg = t3d.make_run_cfg(L, 1, w.p, w.q, w.seed, S, bp_chunk_samples=25024, **kw)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    counts = torch.zeros(8, dtype=torch.int64, device=dev())
    batch = t3d.make_batch([dict(L=L, n_samples=S, e=e, mask=mask, counts8=counts)])
    work = torch.empty(t3d.toric3d_run_batch_workspace_bytes(cfg, batch), dtype=torch.uint8, device=dev())
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        t3d.toric3d_autotune_batch(cfg, batch, work, stream=stream)
        t3d.toric3d_run_batch(cfg, batch, work, stream=stream)
    stream.synchronize()
    got_counts = counts.cpu().numpy()
    assert got_counts.sum() == S
    m = mask.cpu().numpy()
    assert np.array_equal(np.bincount(m, minlength=8), got_counts)

    ocfg = oracle.make_cfg(L, 1, w.p, w.q, w.seed, **kw)
    checked = 0
    # samples only (BP writes its decisions for a chunk's samples, not for the padding lanes of
    # the last word); a sample is skipped when any of its 98,304 posteriors lies within 1e-4 of
    # zero, which happens in roughly half of them; 20 candidates leave enough checked ones
    for i in (0, 1, 2, 63, 64, 65, 127, 25023, 25024, 25025, 50_000, 50_047, 50_048, 77_777, 88_888,
              99_900, 99_935, S - 3, S - 2, S - 1):
        e0 = oracle.noise_batch(L, np.zeros((1, n), np.uint8), w.p, w.seed, i, 1)
        s0 = oracle.measure_batch(L, e0, w.q, w.seed, i, 1)
        _, llr = oracle.bp_batch(L, s0, w.p, w.q, True, w.bp_iters)
        if not (np.abs(llr) > 1e-4).all():
            continue                          # a BP decision within FP32 reach of zero
        ora_mask, ora_e = oracle.run_batch(ocfg, i, 1)
        assert np.array_equal(_sample_bits(e, i), ora_e[0]), i
        assert m[i] == ora_mask[0], i
        checked += 1
    assert checked >= 6


def _word_bits(words: torch.Tensor, w: int) -> np.ndarray:
    """[64][n] bits of the 64 samples of word w of a bit-sliced [n][W] tensor."""
    col = words[:, w].cpu().numpy().view(np.uint64)
    return ((col[None, :] >> np.arange(64, dtype=np.uint64)[:, None]) & np.uint64(1)).astype(np.uint8)


def test_bp_step_full_chunk_L32_per_iteration():
    """toric3d_bp_step over one whole benchmark chunk (L = 32, 25,024 samples =
    391 words, 39.4 GB per message buffer): words 0, 195 and 390 compared with
    the FP64 oracle at iteration 1 (from the priors) and at iterations 8 and 16
    (the oracle seeded with the GPU's messages of the iteration before), at the
    tolerance of the small-lattice per-iteration test."""
    L, S, p = 32, 25024, 0.04
    n, W = inp.n_bits(L), inp.words_for(S)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s = torch.empty_like(e)
    # the benchmark's first-cycle syndrome, plus the residual of a few decoded cycles' worth
    # of noise so BP sees clusters as well as isolated checks
    for t in (1, 2, 3):
        t3d.toric3d_noise(L, e, p, 11, 0, t)
    t3d.toric3d_syndrome(L, e, s, p, 11, 0, 3)
    nfl = t3d.toric3d_bp_message_bytes(L, S) // 4
    A = torch.empty(nfl, dtype=torch.float32, device=dev())
    B = torch.empty(nfl, dtype=torch.float32, device=dev())
    words = (0, 195, 390)
    fe, _ = oracle.incidence(L)
    idx = message_index(L, fe)
    per_word = n * 4 * 64
    sb = {w: _word_bits(s, w) for w in words}

    def snap(buf):
        return {w: gpu_messages_to_oracle(buf[w * per_word:(w + 1) * per_word], L, 64, idx) for w in words}

    l0 = float(np.log((1 - p) / p))
    pool = spawn_pool()
    try:
        t3d.toric3d_bp_step(L, S, s, p, p, None, A)
        checks = {1: (None, snap(A))}
        prev = checks[1][1]
        for it in range(2, 17):
            t3d.toric3d_bp_step(L, S, s, p, p, A, B)
            A, B = B, A
            if it in (8, 16):
                checks[it] = (prev, snap(A))
            if it in (7, 15):
                prev = snap(A)
        for it, (m_prev, m_now) in checks.items():
            for w in words:
                args = [(L, sb[w][i], p, p, None if m_prev is None else m_prev[w][i]) for i in range(64)]
                ref = np.stack(pool.map(bp_messages, args))
                bound = 0.0 if m_prev is None else _input_rounding_bound(m_prev[w], fe, l0)
                bad = np.abs(m_now[w] - ref) > _tol(ref, bound)
                assert not bad.any(), f"iteration {it}, word {w}: {int(bad.sum())} messages out of tolerance"
    finally:
        pool.close()
        pool.join()


def test_bp_pflip_L32_four_cycles_replayed_at_chunk_boundaries():
    """Four cycles of the benchmark's decoder (BP16 with measurement variables,
    then 32 x PFFPFF) on all 10^5 samples with BP in 25,024-sample chunks,
    replayed against the oracle on 64 lanes at and around the chunk boundaries:
    noise, measurement and the schedule bit-exact, BP decisions (read from the
    change of e) equal wherever the oracle's |l| > 1e-4, and the oracle takes
    the GPU's BP decisions so every cycle starts from the same state."""
    w = inp.WORKLOADS["bp_pflip_L32"]
    L, S, p, seed = w.L, w.n_samples, w.p, w.seed
    n, W = inp.n_bits(L), inp.words_for(S)
    chunk = 25024
    lanes = sorted({x for b in (0, chunk, 2 * chunk, 3 * chunk, S - 64)
                    for x in range(max(0, b - 6), min(S, b + 7))} | {S - 1})[:64]
    cols = sorted({i // 64 for i in lanes})
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s = torch.empty_like(e)
    work = torch.empty(t3d.toric3d_bp_workspace_bytes(L, chunk), dtype=torch.uint8, device=dev())
    fwork = torch.empty(t3d.toric3d_flip_workspace_bytes(L, W), dtype=torch.uint8, device=dev())

    def lane_bits(x):
        got = {c: _word_bits(x, c) for c in cols}
        return np.stack([got[i // 64][i % 64] for i in lanes])

    ora_e = np.zeros((len(lanes), n), np.uint8)
    pool = spawn_pool()
    ambiguous = 0
    try:
        for t in range(1, 5):
            t3d.toric3d_noise(L, e, p, seed, 0, t)
            t3d.toric3d_syndrome(L, e, s, w.q, seed, 0, t)
            ora_s = np.empty_like(ora_e)
            for k, i in enumerate(lanes):
                ora_e[k] = oracle.noise_batch(L, ora_e[k:k + 1], p, seed, i, t)[0]
                ora_s[k] = oracle.measure_batch(L, ora_e[k:k + 1], w.q, seed, i, t)[0]
            e_before = lane_bits(e)
            assert np.array_equal(e_before, ora_e) and np.array_equal(lane_bits(s), ora_s)
            t3d.toric3d_bp(L, S, e, s, p, w.q, w.bp_iters, work)
            d = lane_bits(e) ^ e_before
            ref = np.stack(pool.map(bp_llr, [(L, ora_s[k], p, w.q, w.bp_iters) for k in range(len(lanes))]))
            clear = np.abs(ref) > 1e-4
            ambiguous += int((~clear).sum())
            assert np.array_equal(d.astype(bool)[clear], (ref < 0)[clear]), f"cycle {t}: BP decisions differ"
            ora_e ^= d
            ora_s ^= oracle.syndrome_batch(L, d)
            assert np.array_equal(lane_bits(s), ora_s)
            t3d.toric3d_pflip(L, e, s, w.schedule, w.n_apply, 0, seed, 0, t, fwork)
            for k, i in enumerate(lanes):
                ek, sk = ora_e[k:k + 1], ora_s[k:k + 1]
                for a in range(w.n_apply):
                    ek, sk = oracle.flip_batch(L, ek, sk, w.schedule[a % len(w.schedule)] == "P", seed, i, t, a)
                ora_e[k], ora_s[k] = ek[0], sk[0]
            assert np.array_equal(lane_bits(e), ora_e) and np.array_equal(lane_bits(s), ora_s), f"cycle {t}"
    finally:
        pool.close()
        pool.join()
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, S, e, mask)
    assert np.array_equal(mask.cpu().numpy()[lanes], oracle.logical_batch(L, ora_e))
    print(f"ambiguous BP lanes (|l| <= 1e-4) over 4 cycles: {ambiguous}")
