"""The throughput workload at full size, in the launch configuration the
benchmark times: L = 32, p = q = 4%, 10^5 samples, one code cycle of BP16 +
32 x PFFPFF through toric3d_run_batch (BP in chunks of 25,024 samples, after
the BP autotuner has run).  Sampled samples are recomputed one by one by the
oracle; the whole batch is checked by properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev

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
    # S .. 64 W - 1 are the padding lanes of the last word: decoded like any sample (their own
    # keys), left out of the readout
    for i in (0, 1, 63, 64, 25023, 25024, 77_777, S - 1, S):
        e0 = oracle.noise_batch(L, np.zeros((1, n), np.uint8), w.p, w.seed, i, 1)
        s0 = oracle.measure_batch(L, e0, w.q, w.seed, i, 1)
        _, llr = oracle.bp_batch(L, s0, w.p, w.q, True, w.bp_iters)
        if not (np.abs(llr) > 1e-4).all():
            continue                          # a BP decision within FP32 reach of zero
        ora_mask, ora_e = oracle.run_batch(ocfg, i, 1)
        assert np.array_equal(_sample_bits(e, i), ora_e[0]), i
        if i < S:
            assert m[i] == ora_mask[0], i
        checked += 1
    assert checked >= 6
