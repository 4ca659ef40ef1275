"""Pins of the oracle's BP with meta-checks (Sec. 4.1, last paragraph): the
cube / face incidence, the meta-syndrome, BP with one prior per variable
against brute-force marginals and against the pinned BP with degree-1
measurement variables, and its decision on an isolated measurement error."""
import itertools

import numpy as np
import pytest

import oracle
import toric3d_inputs as inp


@pytest.mark.parametrize("L", [2, 3, 4])
def test_every_face_bounds_two_cubes(L):
    n = 3 * L ** 3
    seen = np.zeros(n, dtype=int)
    for c in range(L ** 3):
        fc = oracle.cube_faces(L, c)
        assert len(set(fc.tolist())) == 6
        seen[fc] += 1
    assert (seen == 2).all()


@pytest.mark.parametrize("L", [3, 4, 5])
def test_meta_syndrome_vanishes_on_error_syndromes(L):
    """Error syndromes are closed loops: every cube's six faces have even parity."""
    e = inp.random_bits(20, 3 * L ** 3, 0.1, L)
    for row in e:
        assert not oracle.meta_syndrome(L, oracle.syndrome(L, row)).any()


def test_measurement_error_toggles_its_two_cubes():
    L = 4
    s = oracle.syndrome(L, inp.random_bits(1, 3 * L ** 3, 0.1, 3)[0])
    for f in (0, 17, 3 * L ** 3 - 1):
        s2 = s.copy()
        s2[f] ^= 1
        diff = np.nonzero(oracle.meta_syndrome(L, s2) ^ oracle.meta_syndrome(L, s))[0]
        assert sorted(diff.tolist()) == sorted(c for c in range(L ** 3) if f in oracle.cube_faces(L, c))


def _brute_marginals(nv, checks, syn, prior):
    w0 = np.zeros(nv)
    w1 = np.zeros(nv)
    for x in itertools.product((0, 1), repeat=nv):
        if any(sum(x[v] for v in c) % 2 != syn[i] for i, c in enumerate(checks)):
            continue
        w = np.exp(-sum(prior[v] for v in range(nv) if x[v]))
        for v in range(nv):
            (w1 if x[v] else w0)[v] += w
    return np.log(w0 / w1)


def test_bp_priors_is_exact_on_a_tree():
    """A tree factor graph with different priors: BP's posteriors are the exact marginals."""
    checks = [[0, 1, 2], [2, 3], [3, 4, 5], [1, 6]]
    prior = np.array([2.0, 1.1, 0.7, 3.0, 1.9, 0.4, 2.5])
    cptr = np.cumsum([0] + [len(c) for c in checks]).astype(np.int32)
    cvar = np.array([v for c in checks for v in c], dtype=np.int32)
    for syn in itertools.product((0, 1), repeat=len(checks)):
        llr = oracle.bp_priors(cptr, cvar, np.array(syn, dtype=np.uint8), prior, 12)
        assert np.allclose(llr, _brute_marginals(len(prior), checks, syn, prior), atol=1e-9)


def test_bp_priors_reduces_to_degree_one_measurement_variables():
    """Faces with their measurement variables written out (degree 1, no meta-checks)
    give exactly the pinned BP whose checks carry the constant factor tanh(lq/2)."""
    L, p, q, iters = 3, 0.05, 0.03, 7
    n = 3 * L ** 3
    fe, _ = oracle.incidence(L)
    cptr = np.arange(0, 5 * n + 1, 5, dtype=np.int32)
    cvar = np.concatenate([fe, np.arange(n, 2 * n)[:, None]], axis=1).astype(np.int32).ravel()
    prior = np.r_[np.full(n, np.log((1 - p) / p)), np.full(n, np.log((1 - q) / q))]
    s = inp.random_bits(3, n, 0.2, 8)
    _, ref = oracle.bp_batch(L, s, p, q, True, iters)
    for i in range(3):
        llr = oracle.bp_priors(cptr, cvar, s[i], prior, iters)
        assert np.allclose(llr[:n], ref[i], rtol=1e-12, atol=1e-12)


def test_meta_bp_flags_an_isolated_measurement_error():
    """No qubit error and one wrong outcome: the meta-checks point at the measurement
    variable (negative posterior), no qubit is corrected."""
    L, p, q = 4, 0.04, 0.04
    n = 3 * L ** 3
    e = np.zeros((1, n), dtype=np.uint8)
    s = np.zeros((1, n), dtype=np.uint8)
    f = 37
    s[0, f] = 1
    e2, s2, llr = oracle.bp_meta_decode_batch(L, e, s, p, q, 10)
    assert not e2.any() and np.array_equal(s2, s)
    meas = llr[0, n:]
    assert meas[f] < 0 and (np.delete(meas, f) > 0).all()
    assert (llr[0, :n] > 0).all()


def test_bp_priors_from_resumes_exactly():
    """k iterations, then m more from the returned messages, equal k + m iterations."""
    L, p, q = 3, 0.05, 0.04
    n = 3 * L ** 3
    cptr, cvar = oracle.meta_tanner(L)
    s = inp.random_bits(1, n, 0.15, 12)[0]
    syn = np.r_[s, oracle.meta_syndrome(L, s)]
    prior = np.r_[np.full(n, np.log((1 - p) / p)), np.full(n, np.log((1 - q) / q))]
    llr7, cv7 = oracle.bp_priors_from(cptr, cvar, syn, prior, 7)
    assert np.array_equal(llr7, oracle.bp_priors(cptr, cvar, syn, prior, 7))
    _, cv3 = oracle.bp_priors_from(cptr, cvar, syn, prior, 3)
    llr34, cv34 = oracle.bp_priors_from(cptr, cvar, syn, prior, 4, cv3)
    assert np.array_equal(llr34, llr7) and np.array_equal(cv34, cv7)
    assert np.array_equal(oracle.bp_priors_from(cptr, cvar, syn, prior, 0, cv7)[1], cv7)


def test_meta_tanner_shape():
    L = 3
    n = 3 * L ** 3
    cptr, cvar = oracle.meta_tanner(L)
    assert len(cptr) == n + L ** 3 + 1 and cptr[-1] == 5 * n + 6 * L ** 3
    assert (np.diff(cptr)[:n] == 5).all() and (np.diff(cptr)[n:] == 6).all()
    assert (cvar[cptr[n]:] >= n).all()


def test_run_with_meta_checks_uses_them():
    """A whole run with bp_meta decodes every cycle with BP + meta-checks: the same
    cycle assembled from the oracle's single steps gives the same final error."""
    L, T, p = 3, 2, 0.04
    cfg = oracle.make_cfg(L, T, p, p, 5, use_bp=True, bp_iters=5, bp_meta=True, schedule="PFF", n_apply=3)
    _, e_run = oracle.run_batch(cfg, 0, 3)
    for sample in range(3):
        e = np.zeros(3 * L ** 3, dtype=np.uint8)
        for t in (1, 2):
            e = oracle.noise(L, e, p, 5, sample, t)
            s = oracle.measure(L, e, p, 5, sample, t)
            e2, s2, _ = oracle.bp_meta_decode_batch(L, e[None], s[None], p, p, 5)
            e, s = e2[0], s2[0]
            for k, kind in enumerate("PFF"):
                if kind == "P":
                    e, s = oracle.pflip_once(L, e, s, seed=5, sample=sample, cycle=t, sweep=k)
                else:
                    e, s = oracle.flip_once(L, e, s)
        assert np.array_equal(e, e_run[sample])
