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


def run_sample_if_clear(args):
    """One sample of a one-cycle BP + p-flip run recomputed by the oracle: (i, e bits, mask),
    or None when one of the sample's first-cycle BP posteriors lies within 1e-4 of zero (a
    decision FP32 and FP64 may take differently)."""
    L, p, q, seed, i, iters, kw = args
    n = 3 * L ** 3
    e0 = oracle.noise_batch(L, np.zeros((1, n), np.uint8), p, seed, i, 1)
    s0 = oracle.measure_batch(L, e0, q, seed, i, 1)
    _, llr = oracle.bp_batch(L, s0, p, q, True, iters)
    if not (np.abs(llr) > 1e-4).all():
        return None
    mask, e = oracle.run_batch(oracle.make_cfg(L, 1, p, q, seed, **kw), i, 1)
    return i, e[0], int(mask[0])


def run_range(args):
    """Samples [s0, s0 + n) of a run without BP recomputed by the oracle: (s0, mask, e bits)."""
    L, T, p, q, seed, kw, s0, n = args
    mask, e = oracle.run_batch(oracle.make_cfg(L, T, p, q, seed, **kw), s0, n)
    return s0, mask, e
