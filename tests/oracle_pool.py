"""Oracle work on one sample at a time for the process pools of the full-size
GPU tests.  Pools must use the 'spawn' start method (a process forked after
the first CUDA call can hang)."""
from __future__ import annotations

import multiprocessing
import os

import numpy as np

import oracle


def spawn_pool(max_procs: int = 16):
    return multiprocessing.get_context("spawn").Pool(max(1, min(max_procs, os.cpu_count() or 1)))


def bp_llr(args):
    """Posteriors of `iters` BP iterations from the priors on one syndrome."""
    L, s_bits, p, q, iters = args
    _, llr = oracle.bp_batch(L, s_bits[None, :], p, q, True, iters)
    return llr[0]


def bp_messages(args):
    """Check->variable messages of one iteration started from m_in (None: the priors)."""
    L, s_bits, p, q, m_in = args
    m, _ = oracle.bp_batch(L, s_bits[None, :], p, q, True, 1, m_in=None if m_in is None else m_in[None, :])
    return m[0]
