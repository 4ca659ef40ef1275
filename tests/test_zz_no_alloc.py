"""toric3d_flip_noalloc: the flip decoder for callers that cannot give the
library device memory (a decoder in a control loop with memory fixed at
start-up, a plugin whose host application owns all device allocations, a
caller that cannot risk the synchronisation cudaMalloc may cause).  Its
scratch is a fixed array inside the library.  The test calls it through the C
ABI twice in a row -- the second call on the first call's output, so the
shared scratch starts with stale contents -- and checks each result bit for
bit against toric3d_flip given a separate workspace.  This file is collected
last on purpose."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu


def _noisy(L, S, seed):
    n = 3 * L ** 3
    e = inp.random_bits(S, n, 0.05, seed)
    return e, oracle.syndrome_batch(L, e) ^ inp.random_bits(S, n, 0.03, seed + 1)


@pytest.mark.parametrize("L,S,sweeps", [(8, 2000, 3), (5, 130, 4)])
def test_noalloc_flip_matches_workspace_flip_on_two_calls(L, S, sweeps):
    ebits, sbits = _noisy(L, S, seed=L)
    e_ref, s_ref = upload_bits(ebits), upload_bits(sbits)
    e_na, s_na = upload_bits(ebits), upload_bits(sbits)
    work = workspace(t3d.toric3d_flip_workspace_bytes(L, e_ref.shape[1]))
    for call in range(2):
        t3d.toric3d_flip(L, e_ref, s_ref, sweeps, work)
        t3d.toric3d_flip_noalloc(L, e_na, s_na, sweeps)
        torch.cuda.synchronize()
        assert np.array_equal(download_bits(e_na, S), download_bits(e_ref, S)), call
        assert np.array_equal(download_bits(s_na, S), download_bits(s_ref, S)), call


def test_noalloc_flip_rejects_sizes_beyond_its_scratch():
    L, words = 32, 64            # 3 * 32^3 * 64 * 8 bytes = 48 MiB > 32 MiB
    e = torch.zeros((3 * L ** 3, words), dtype=torch.int64, device="cuda")
    s = torch.zeros_like(e)
    with pytest.raises(t3d.T3DError, match="built-in scratch"):
        t3d.toric3d_flip_noalloc(L, e, s, 1)


def test_noalloc_flip_replayed_from_a_captured_graph():
    # the use the entry point exists for: after one eager call (which looks up the scratch
    # address outside any capture), a call captured on a side stream into a CUDA graph and
    # replayed, each replay checked against toric3d_flip with a workspace
    L, S, sweeps = 6, 500, 3
    ebits, sbits = _noisy(L, S, seed=11)
    e_ref, s_ref = upload_bits(ebits), upload_bits(sbits)
    e_na, s_na = upload_bits(ebits), upload_bits(sbits)
    work = workspace(t3d.toric3d_flip_workspace_bytes(L, e_ref.shape[1]))
    t3d.toric3d_flip(L, e_ref, s_ref, 1, work)
    t3d.toric3d_flip_noalloc(L, e_na, s_na, 1)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        t3d.toric3d_flip_noalloc(L, e_na, s_na, sweeps, stream=side)
    torch.cuda.synchronize()
    # capturing ran nothing: the states still match after the eager call
    assert np.array_equal(download_bits(e_na, S), download_bits(e_ref, S))
    for replay in range(2):
        graph.replay()
        t3d.toric3d_flip(L, e_ref, s_ref, sweeps, work)
        torch.cuda.synchronize()
        assert np.array_equal(download_bits(e_na, S), download_bits(e_ref, S)), replay
        assert np.array_equal(download_bits(s_na, S), download_bits(s_ref, S)), replay
