"""Whole-run semantics of the oracle (Sec. 3.1 Fig. 2, Sec. 3.2 schedule list,
Sec. 4.2 p-BP): determinism, independence of samples, exact resumption, and
the noiseless final round."""
import numpy as np
import pytest

import oracle


def _cfg(**kw):
    base = dict(L=4, T=4, p=0.02, q=0.02, seed=3, schedule="FFPFF")
    base.update(kw)
    return oracle.make_cfg(**base)


def test_no_noise_means_no_error():
    for kw in (dict(schedule="F"), dict(schedule="PFFPFF", use_bp=True, bp_iters=5)):
        cfg = _cfg(p=0.0, q=0.0, **kw)
        m, e = oracle.run_sample(cfg, 5)
        assert m == 0 and e.sum() == 0


@pytest.mark.parametrize("kw", [dict(schedule="F", n_apply=3), dict(schedule="FFPFF"),
                                dict(schedule="PFFPFF", use_bp=True, bp_iters=6)])
def test_batch_equals_per_sample_runs(kw):
    cfg = _cfg(**kw)
    mask, e = oracle.run_batch(cfg, 64, 6)
    for i in range(6):
        m1, e1 = oracle.run_sample(cfg, 64 + i)
        assert m1 == mask[i] and np.array_equal(e1, e[i])


@pytest.mark.parametrize("kw", [dict(schedule="FFPFF"), dict(schedule="PFFPFF", use_bp=True, bp_iters=4)])
def test_split_run_resumes_exactly(kw):
    full = _cfg(T=6, **kw)
    first = _cfg(T=3, **kw)
    second = _cfg(T=3, cycle0=3, **kw)
    for sample in (0, 1, 130):
        m_full, e_full = oracle.run_sample(full, sample)
        _, e_half = oracle.run_sample(first, sample)
        m2, e2 = oracle.run_sample(second, sample, e_half)
        assert m2 == m_full and np.array_equal(e2, e_full)


def test_perfect_round_clears_syndrome_and_lines_are_unanimous():
    cfg = _cfg(p=0.01, q=0.01, T=4, schedule="F", n_apply=32, perfect_round=True,
               perfect_max_sweeps=32)
    mask, e = oracle.run_batch(cfg, 0, 40)
    cleared = 0
    for i in range(40):
        if oracle.syndrome(4, e[i]).sum() == 0:
            cleared += 1
            m, counts = oracle.logical(4, e[i])
            assert all(c in (0, 16) for c in counts) and m == mask[i]
    assert cleared >= 36


def test_schedule_string_is_cycled_for_n_apply():
    # "PF" cycled over 3 applications must equal "PFP" once
    a = oracle.run_batch(_cfg(schedule="PF", n_apply=3), 0, 8)
    b = oracle.run_batch(_cfg(schedule="PFP"), 0, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
