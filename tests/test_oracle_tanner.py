"""Pins of the oracle's decoders on generic Tanner graphs (the question of
Sec. 5: do these decoders carry over to other LDPC codes?).  On the 3D toric
code's own Tanner graph they must reproduce the toric oracle, which is pinned
against the paper; the p-flip coin follows its stated key; the hypergraph
product of two cyclic repetition codes is the 2D toric code, where single
errors are fixed in one application."""
import numpy as np
import pytest

import oracle
import toric3d_inputs as inp


def _dense(cptr, cvar, n):
    H = np.zeros((len(cptr) - 1, n), dtype=np.int64)
    for c in range(len(cptr) - 1):
        H[c, cvar[cptr[c]:cptr[c + 1]]] = 1
    return H


@pytest.mark.parametrize("L", [3, 4])
def test_toric_graph_reproduces_toric_oracle(L):
    n = 3 * L ** 3
    cptr, cvar = oracle.toric_tanner(L)
    e = inp.random_bits(40, n, 0.08, L)
    assert np.array_equal(oracle.tanner_syndrome_batch(cptr, cvar, e), oracle.syndrome_batch(L, e))
    e1 = oracle.tanner_noise_batch(e, 0.05, 7, 64, 3)
    assert np.array_equal(e1, oracle.noise_batch(L, e, 0.05, 7, 64, 3))
    s1 = oracle.tanner_measure_batch(cptr, cvar, e1, 0.05, 7, 64, 3)
    assert np.array_equal(s1, oracle.measure_batch(L, e1, 0.05, 7, 64, 3))
    ef, sf = oracle.tanner_rule_batch(cptr, cvar, e1, s1)
    ef_ref, sf_ref = oracle.flip_batch(L, e1, s1)
    assert np.array_equal(ef, ef_ref) and np.array_equal(sf, sf_ref)


@pytest.mark.parametrize("code", ["toric", "hgp"])
def test_pflip_flips_majority_and_coin_chosen_ties(code):
    """p-flip = the majority variables plus the tie variables whose coin (word v mod 4
    of the coin stream keyed v / 4) is 1; counts from the dense parity-check matrix."""
    if code == "toric":
        cptr, cvar = oracle.toric_tanner(3)
        n = 81
    else:
        cptr, cvar, n = inp.hgp_workload(8, 3)
    H = _dense(cptr, cvar, n)
    e = inp.random_bits(70, n, 0.1, 5)
    s = oracle.tanner_syndrome_batch(cptr, cvar, e) ^ inp.random_bits(70, len(cptr) - 1, 0.05, 6)
    seed, sample0, cycle, sweep = 11, 64, 2, 3
    e2, s2 = oracle.tanner_rule_batch(cptr, cvar, e, s, True, seed, sample0, cycle, sweep)
    deg = H.sum(axis=0)
    ties_seen = 0
    for i in range(len(e)):
        unsat = H.T @ s[i]
        maj = 2 * unsat > deg
        tie = 2 * unsat == deg
        coin = np.array([oracle.tanner_coin(seed, v, cycle, sweep, sample0 + i) for v in range(n)], dtype=bool)
        f = maj | (tie & coin)
        ties_seen += int(tie.sum())
        assert np.array_equal(e2[i] ^ e[i], f.astype(np.uint8))
        assert np.array_equal(s2[i] ^ s[i], (H @ f % 2).astype(np.uint8))
    assert ties_seen > 0


def test_coin_key():
    """The coin of variable v is word v mod 4 of the coin stream keyed by site v / 4."""
    for v in (0, 1, 2, 3, 4, 7, 1001):
        for sample in (0, 5, 63, 64, 200):
            assert oracle.tanner_coin(9, v, 4, 2, sample) == oracle.lib().t3o_coin(9, v // 4, v % 4, 4, 2, sample)


def test_hgp_of_cycles_is_the_2d_toric_code():
    L = 5
    X, Z, n = inp.hypergraph_product(inp.cyclic_repetition(L), L, inp.cyclic_repetition(L), L)
    assert n == 2 * L * L and len(X) == len(Z) == L * L
    cptr, cvar = inp.csr(Z)
    H = _dense(cptr, cvar, n)
    assert (H.sum(axis=1) == 4).all() and (H.sum(axis=0) == 2).all()
    HX = _dense(*inp.csr(X), n)
    assert not (HX @ H.T % 2).any()
    # every single error is removed by one flip application (both its checks unsatisfied,
    # every other qubit sees at most one)
    e = np.eye(n, dtype=np.uint8)
    s = oracle.tanner_syndrome_batch(cptr, cvar, e)
    e2, s2 = oracle.tanner_rule_batch(cptr, cvar, e, s)
    assert not e2.any() and not s2.any()


def test_hgp_workload_structure():
    cptr, cvar, n = inp.hgp_workload(40, 1)
    m = len(cptr) - 1
    assert n == 40 * 40 + 30 * 30 and m == 40 * 30
    assert (np.diff(cptr) == 7).all()
    deg = np.bincount(cvar, minlength=n)
    assert set(deg.tolist()) == {3, 4}
    X, Z, _ = inp.hypergraph_product(inp.random_biregular(40, 30, 3, 4, 1), 40,
                                     inp.random_biregular(40, 30, 3, 4, 2), 40)
    assert not (_dense(*inp.csr(X), n) @ _dense(cptr, cvar, n).T % 2).any()


def test_bp_on_toric_graph_equals_toric_bp():
    """Per-variable priors l0 on the toric graph without measurement variables: the
    generic BP's posteriors equal the toric BP's, and the decision is applied."""
    L, p, iters = 3, 0.05, 8
    n = 3 * L ** 3
    cptr, cvar = oracle.toric_tanner(L)
    e = inp.random_bits(6, n, 0.06, 2)
    s = oracle.syndrome_batch(L, e)
    e2, s2, llr = oracle.tanner_bp_batch(cptr, cvar, e, s, np.full(n, np.log((1 - p) / p)), iters)
    _, ref = oracle.bp_batch(L, s, p, 0.0, False, iters)
    assert np.allclose(llr, ref, rtol=1e-12, atol=1e-12)
    d = (llr < 0).astype(np.uint8)
    assert np.array_equal(e2, e ^ d) and np.array_equal(s2, s ^ oracle.syndrome_batch(L, d))
