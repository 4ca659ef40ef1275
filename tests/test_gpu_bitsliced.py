"""Bit-exact parity of the bit-sliced CUDA kernels with the oracle: layout
conversion, qubit noise, noisy syndrome, flip / p-flip applications and the
logical readout, through the C ABI.  Includes the exhaustive L = 2 checks
(all 2^24 error patterns for the syndrome and the readout, all 2^24 syndrome
patterns for one flip and one p-flip application) and ragged sample counts."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace, zeros_words

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("S", [1, 63, 64, 65, 1000])
def test_pack_unpack_roundtrip(S):
    bits = inp.random_bits(S, 37, 0.3, seed=S)
    b = torch.from_numpy(bits).to(dev())
    W = inp.words_for(S)
    words = torch.full((37, W), -1, dtype=torch.int64, device=dev())
    t3d.toric3d_pack(37, S, b, words)
    assert np.array_equal(words.cpu().numpy().view(np.uint64), inp.pack(bits))
    back = torch.zeros_like(b)
    t3d.toric3d_unpack(37, S, words, back)
    assert np.array_equal(back.cpu().numpy(), bits)


@pytest.mark.parametrize("L,S,p,sample0,cycle", [(2, 64, 0.3, 0, 1), (3, 1000, 0.04, 128, 7),
                                                 (4, 130, 0.01, 640, 2), (5, 257, 0.5, 0, 3),
                                                 (4, 100, 1.0, 64, 1), (4, 100, 0.0, 0, 1)])
def test_noise_matches_oracle(L, S, p, sample0, cycle):
    n = 3 * L ** 3
    start = inp.random_bits(S, n, 0.1, seed=L + S)
    e = upload_bits(start)
    t3d.toric3d_noise(L, e, p, 99, sample0, cycle)
    want = oracle.noise_batch(L, start, p, 99, sample0, cycle)
    assert np.array_equal(download_bits(e, S), want)


@pytest.mark.parametrize("L,S,q", [(2, 100, 0.0), (3, 333, 0.04), (4, 1000, 0.02), (6, 70, 0.2)])
def test_syndrome_matches_oracle(L, S, q):
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, 0.15, seed=L)
    e = upload_bits(ebits)
    s = zeros_words(n, S)
    t3d.toric3d_syndrome(L, e, s, q, 5, 64, 3)
    want = oracle.measure_batch(L, ebits, q, 5, 64, 3)
    assert np.array_equal(download_bits(s, S), want)


@pytest.mark.parametrize("L,S,schedule,n_apply,sweep0", [(3, 200, "F", 1, 0), (4, 500, "FFPFF", 5, 0),
                                                         (4, 130, "PF", 7, 3), (5, 64, "P", 2, 1),
                                                         (6, 100, "FFPFF", 4, 0)])
def test_sweeps_match_oracle(L, S, schedule, n_apply, sweep0):
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, 0.05, seed=L)
    meas = inp.random_bits(S, n, 0.04, seed=L + 1)
    sbits = oracle.syndrome_batch(L, ebits) ^ meas
    e, s = upload_bits(ebits), upload_bits(sbits)
    work = workspace(t3d.toric3d_flip_workspace_bytes(L, e.shape[1]))
    seed, sample0, cycle = 17, 192, 4
    t3d.toric3d_pflip(L, e, s, schedule, n_apply, sweep0, seed, sample0, cycle, work)
    we, ws = ebits, sbits
    for k in range(n_apply):
        we, ws = oracle.flip_batch(L, we, ws, schedule[k % len(schedule)] == "P", seed, sample0, cycle,
                                   sweep0 + k)
    assert np.array_equal(download_bits(e, S), we)
    assert np.array_equal(download_bits(s, S), ws)


def test_plain_flip_entry_point():
    L, S = 4, 300
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, 0.04, seed=1)
    sbits = oracle.syndrome_batch(L, ebits)
    e, s = upload_bits(ebits), upload_bits(sbits)
    t3d.toric3d_flip(L, e, s, 3, workspace(t3d.toric3d_flip_workspace_bytes(L, e.shape[1])))
    we, ws = ebits, sbits
    for _ in range(3):
        we, ws = oracle.flip_batch(L, we, ws)
    assert np.array_equal(download_bits(e, S), we) and np.array_equal(download_bits(s, S), ws)


@pytest.mark.parametrize("L,S,density", [(2, 200, 0.4), (3, 500, 0.3), (4, 1000, 0.45), (5, 99, 0.5),
                                         (8, 130, 0.5), (6, 5000, 0.45), (16, 700, 0.5)])
def test_logical_matches_oracle(L, S, density):
    # 5000 samples: 79 words, ten word tiles with a ragged last one; L = 16: 256 lines per axis
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, density, seed=L)
    e = upload_bits(ebits)
    mask = torch.zeros(S, dtype=torch.uint8, device=dev())
    counts = torch.full((8,), -5, dtype=torch.int64, device=dev())
    t3d.toric3d_logical(L, S, e, mask, counts)
    want = oracle.logical_batch(L, ebits)
    got = mask.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.array_equal(counts.cpu().numpy(), np.bincount(want, minlength=8))
    assert len(set(got.tolist())) > 1


# ------------------------------------------------------------------ exhaustive L = 2
CHUNK = 1 << 22


def _pattern_chunk(start):
    idx = np.arange(start, start + CHUNK, dtype=np.int64)
    return ((idx[:, None] >> np.arange(24, dtype=np.int64)[None, :]) & 1).astype(np.uint8)


@pytest.mark.parametrize("start", range(0, 1 << 24, CHUNK))
def test_exhaustive_L2_syndrome_and_logical(start):
    L = 2
    bits = _pattern_chunk(start)
    e = upload_bits(bits)
    s = zeros_words(24, CHUNK)
    t3d.toric3d_syndrome(L, e, s, 0.0, 0, 0, 1)
    assert np.array_equal(download_bits(s, CHUNK), oracle.syndrome_batch(L, bits))
    mask = torch.zeros(CHUNK, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, CHUNK, e, mask)
    assert np.array_equal(mask.cpu().numpy(), oracle.logical_batch(L, bits))


@pytest.mark.parametrize("start", range(0, 1 << 24, CHUNK))
def test_exhaustive_L2_flip_and_pflip_over_all_syndromes(start):
    L = 2
    sbits = _pattern_chunk(start)
    zeros = np.zeros_like(sbits)
    for probabilistic in (False, True):
        e, s = upload_bits(zeros), upload_bits(sbits)
        work = workspace(t3d.toric3d_flip_workspace_bytes(L, e.shape[1]))
        t3d.toric3d_pflip(L, e, s, "P" if probabilistic else "F", 1, 5, 3, start, 2, work)
        we, ws = oracle.flip_batch(L, zeros, sbits, probabilistic, 3, start, 2, 5)
        assert np.array_equal(download_bits(e, CHUNK), we)
        assert np.array_equal(download_bits(s, CHUNK), ws)


# ------------------------------------------------------------------ flip until clear
@pytest.mark.parametrize("L,S,p,max_sweeps", [(4, 1000, 0.01, 32), (6, 3000, 0.02, 32), (8, 200, 0.06, 5),
                                              (33, 64, 0.004, 8)])
def test_flip_until_clear_matches_fixed_sweeps_and_counts_the_sweeps(L, S, p, max_sweeps):
    # L = 33 takes the one-thread-per-site flip kernel, the others the shared-memory one; the
    # (8, 0.06, 5) case does not clear, so every application runs
    n = 3 * L ** 3
    ebits = inp.random_bits(S, n, p, seed=100 + L)
    sbits = oracle.syndrome_batch(L, ebits)
    e_fix, s_fix = upload_bits(ebits), upload_bits(sbits)
    e_stop, s_stop = upload_bits(ebits), upload_bits(sbits)
    W = e_fix.shape[1]
    t3d.toric3d_flip(L, e_fix, s_fix, max_sweeps, workspace(t3d.toric3d_flip_workspace_bytes(L, W)))
    done = torch.full((1,), -7, dtype=torch.int32, device=dev())
    t3d.toric3d_flip_until_clear(L, e_stop, s_stop, max_sweeps,
                                 workspace(t3d.toric3d_flip_until_clear_workspace_bytes(L, W)), done)
    torch.cuda.synchronize()
    assert np.array_equal(download_bits(e_stop, S), download_bits(e_fix, S))
    assert np.array_equal(download_bits(s_stop, S), download_bits(s_fix, S))
    # the oracle's count: applications that start from a syndrome with an unsatisfied check
    we, ws, count = ebits, sbits, 0
    while count < max_sweeps and ws.any():
        we, ws = oracle.flip_batch(L, we, ws)
        count += 1
    assert int(done.item()) == count
    assert np.array_equal(download_bits(e_stop, S), we)


def test_flip_until_clear_on_a_clear_syndrome_runs_no_sweep():
    L, S = 5, 300
    ebits = inp.random_bits(S, 3 * L ** 3, 0.0, seed=3)
    e, s = upload_bits(ebits), upload_bits(ebits)
    done = torch.full((1,), -7, dtype=torch.int32, device=dev())
    t3d.toric3d_flip_until_clear(L, e, s, 16, workspace(t3d.toric3d_flip_until_clear_workspace_bytes(L, e.shape[1])),
                                 done)
    torch.cuda.synchronize()
    assert int(done.item()) == 0
    assert not download_bits(e, S).any() and not download_bits(s, S).any()
