"""Batched runs over lattices of different sizes (one persistent launch per
step for all of them): every item must end exactly where a separate run of
the same ensemble ends, with and without BP chunk rounds, graph replay and
autotuned launch caps."""
import numpy as np
import pytest
import torch

import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, workspace

pytestmark = pytest.mark.gpu

SPECS = [(4, 300, 0), (5, 130, 640), (6, 257, 64), (3, 64, 128)]


def _alloc(L, S):
    n = 3 * L ** 3
    return (torch.zeros((n, inp.words_for(S)), dtype=torch.int64, device=dev()),
            torch.zeros(S, dtype=torch.uint8, device=dev()),
            torch.zeros(8, dtype=torch.int64, device=dev()))


def _single(kw, L, S, sample0):
    e, mask, counts = _alloc(L, S)
    cfg = t3d.make_run_cfg(L, kw["T"], kw["p"], kw["p"], 5, S, sample0=sample0, **kw["dec"])
    t3d.toric3d_run_cycles(cfg, e, workspace(t3d.toric3d_run_workspace_bytes(cfg)), mask, counts)
    torch.cuda.synchronize()
    return download_bits(e, S), mask.cpu().numpy(), counts.cpu().numpy()


def _batch(kw, specs, ws_bytes=None, use_graph=False, tune=False):
    bufs = [_alloc(L, S) for L, S, _ in specs]
    batch = t3d.make_batch([dict(L=L, n_samples=S, sample0=o, e=b[0], mask=b[1], counts8=b[2])
                            for (L, S, o), b in zip(specs, bufs)])
    cfg = t3d.make_run_cfg(8, kw["T"], kw["p"], kw["p"], 5, 1, use_graph=use_graph, **kw["dec"])
    need = t3d.toric3d_run_batch_workspace_bytes(cfg, batch)
    assert need > 0
    work = workspace(ws_bytes or need)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())   # inputs were written on the current stream
    with torch.cuda.stream(stream):
        if tune:
            cap, ms = t3d.toric3d_autotune_batch(cfg, batch, work)
            assert cap in (0, 1, 2, 4, 6, 8) and ms > 0
        t3d.toric3d_run_batch(cfg, batch, work)
    stream.synchronize()
    return [(download_bits(b[0], S), b[1].cpu().numpy(), b[2].cpu().numpy())
            for (L, S, _), b in zip(specs, bufs)]


DECODERS = {
    "flip": dict(T=3, p=0.02, dec=dict(schedule="F", n_apply=4, perfect_round=True, perfect_max_sweeps=8)),
    "pflip": dict(T=3, p=0.03, dec=dict(schedule="FFPFF", n_apply=5)),
    "bp_pflip": dict(T=2, p=0.04, dec=dict(use_bp=True, bp_iters=6, schedule="PFFPFF", n_apply=6)),
}


@pytest.mark.parametrize("name", sorted(DECODERS))
def test_batch_items_equal_separate_runs(name):
    kw = DECODERS[name]
    got = _batch(kw, SPECS)
    for (L, S, o), g in zip(SPECS, got):
        want = _single(kw, L, S, o)
        assert all(np.array_equal(a, b) for a, b in zip(g, want)), (name, L)


def test_batch_bp_chunk_rounds_are_invisible():
    kw = DECODERS["bp_pflip"]
    specs = [(4, 1000, 0), (6, 700, 0)]
    full = _batch(kw, specs)
    cfg = t3d.make_run_cfg(8, 1, 0.04, 0.04, 5, 1, use_bp=True, bp_iters=6, schedule="PFFPFF", n_apply=6)
    # just enough for the two states and one 64-sample word per item: many rounds
    tight = sum(2 * ((3 * L ** 3 * inp.words_for(S) * 8 + 255) // 256 * 256) for L, S, _ in specs)
    tight += sum((2 * 3 * L ** 3 * 4 * 64 * 4 + L ** 3 * 32 + 255) // 256 * 256 for L, _, _ in specs)
    small = _batch(kw, specs, ws_bytes=tight)
    for a, b in zip(full, small):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_batch_graph_replay_and_autotune():
    kw = DECODERS["bp_pflip"]
    a = _batch(kw, SPECS)
    b = _batch(kw, SPECS, use_graph=True, tune=True)
    for x, y in zip(a, b):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    t3d.toric3d_set_blocks_per_sm("bp_step", 0)
