"""The shared-memory flip's tile shapes against the oracle, bit for bit.

A batch whose lattices all have L >= 32 runs tiles of up to 1024 threads (L x Wt,
Wt = 32 words at L = 32, 16 above), a batch with a smaller lattice tiles of at most
256; lattices above the tile limit take the one-thread-per-(site, word) kernel.
These cases cover each shape with a ragged last word tile and a batch whose items
have different tiles (the block takes the largest, the smaller item's extra threads
idle): flip and p-flip schedules over two code cycles (Sec. 3.1, Sec. 3.2), the
error states and the logical masks compared with the oracle on sampled lanes: the
first 16 samples of each item and the last 16 (in its partial last word), recomputed
one by one in a spawn pool."""
import numpy as np
import pytest
import torch

import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, workspace
from oracle_pool import run_range, spawn_pool

pytestmark = pytest.mark.gpu

T, P, SEED = 2, 0.03, 11
DEC = dict(schedule="FFPFF", n_apply=5)


def _alloc(L, S):
    return (torch.zeros((inp.n_bits(L), inp.words_for(S)), dtype=torch.int64, device=dev()),
            torch.zeros(S, dtype=torch.uint8, device=dev()),
            torch.zeros(8, dtype=torch.int64, device=dev()))


def _lanes(S):
    """The first 16 samples and the last 16 (in the partial last word)."""
    return sorted(set(range(min(16, S))) | set(range(max(0, S - 16), S)))


def _check_against_oracle(L, S, sample0, e_bits, mask):
    lanes = _lanes(S)
    with spawn_pool() as pool:
        got = pool.map(run_range, [(L, T, P, P, SEED, DEC, sample0 + i, 1) for i in lanes])
    for i, (s0, ora_mask, ora_e) in zip(lanes, got):
        assert s0 == sample0 + i
        assert np.array_equal(e_bits[i], ora_e[0]), (L, i)
        assert mask[i] == ora_mask[0], (L, i)


@pytest.mark.parametrize("L,S", [(32, 1093), (33, 1093), (40, 1089)])
def test_single_lattice_tiles_match_oracle(L, S):
    # 18 words: L = 32 32-word tiles, the second partial; L = 33 and 40 16-word tiles of 528 and
    # 640 threads (block sizes not a power of two), the second partial
    e, mask, counts = _alloc(L, S)
    cfg = t3d.make_run_cfg(L, T, P, P, SEED, S, **DEC)
    t3d.toric3d_run_cycles(cfg, e, workspace(t3d.toric3d_run_workspace_bytes(cfg)), mask, counts)
    torch.cuda.synchronize()
    m = mask.cpu().numpy()
    assert int(counts.sum()) == S
    _check_against_oracle(L, S, 0, download_bits(e, S), m)


@pytest.mark.parametrize("specs", [[(32, 2100, 0), (36, 1100, 2112)],   # tiles of 1024 and 576 threads
                                   [(32, 1100, 0), (12, 300, 1152)]])  # at most 256 threads (L = 12)
def test_batch_of_tile_shapes_matches_oracle(specs):
    bufs = [_alloc(L, S) for L, S, _ in specs]
    batch = t3d.make_batch([dict(L=L, n_samples=S, sample0=o, e=b[0], mask=b[1], counts8=b[2])
                            for (L, S, o), b in zip(specs, bufs)])
    cfg = t3d.make_run_cfg(8, T, P, P, SEED, 1, **DEC)
    work = workspace(t3d.toric3d_run_batch_workspace_bytes(cfg, batch))
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        t3d.toric3d_run_batch(cfg, batch, work)
    stream.synchronize()
    for (L, S, o), (e, mask, counts) in zip(specs, bufs):
        assert int(counts.sum()) == S
        _check_against_oracle(L, S, o, download_bits(e, S), mask.cpu().numpy())
