"""Multi-replica host logic on CPU (gloo, world size 2): each rank decodes a
disjoint sample range starting at replica_sample0(rank, S); summing the
per-rank logical-outcome histograms must equal one process decoding the
whole range, bit for bit (the generator is keyed by global sample index)."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

L, T, P, S_PER_RANK, SEED = 4, 3, 0.03, 100, 12
KW = dict(schedule="FFPFF")


def _rank_main(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2212_06985_gb300 import replica_sample0
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = oracle.make_cfg(L, T, P, P, SEED, **KW)
    mask, _ = oracle.run_batch(cfg, replica_sample0(rank, S_PER_RANK), S_PER_RANK)
    counts = torch.tensor(np.bincount(mask, minlength=8), dtype=torch.int64)
    dist.all_reduce(counts)
    if rank == 0:
        np.save(out_path, counts.numpy())
    dist.destroy_process_group()


def test_two_replicas_sum_to_one_batch(tmp_path):
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "counts.npy")
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    summed = np.load(out)

    import oracle
    from paper_2212_06985_gb300 import replica_sample0
    cfg = oracle.make_cfg(L, T, P, P, SEED, **KW)
    stride = replica_sample0(1, S_PER_RANK)
    whole, _ = oracle.run_batch(cfg, 0, stride + S_PER_RANK)
    keep = np.r_[0:S_PER_RANK, stride:stride + S_PER_RANK]
    assert np.array_equal(summed, np.bincount(whole[keep], minlength=8))
    assert summed.sum() == 2 * S_PER_RANK


def test_replica_ranges_are_disjoint_and_word_aligned():
    sys.path.insert(0, ROOT)
    from paper_2212_06985_gb300 import replica_sample0
    for S in (1, 64, 100, 100_000):
        starts = [replica_sample0(r, S) for r in range(8)]
        assert all(s % 64 == 0 for s in starts)
        assert all(b - a >= S for a, b in zip(starts, starts[1:]))
