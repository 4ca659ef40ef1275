"""Pins of the oracle's belief propagation (Sec. 4.1, Eqs. 1-4).

* On an acyclic Tanner graph product-sum BP is exact: after enough iterations
  its posterior LLR (Eq. 4) equals the log-odds of the marginal of
  P(e | s), which a brute-force sum over all error patterns gives.  With the
  measurement-error variables of Sec. 4.1 the check factor becomes
  q^[parity != s] (1-q)^[parity == s]; without them it is a hard constraint.
* On the toric graph the first iteration has a closed form: every
  variable->check message is the prior l0 (Eq. 1), so every check->variable
  message is (-1)^{s_f} 2 atanh(tq tanh(l0/2)^3).
* With zero syndrome all messages stay equal by symmetry and follow the scalar
  map m -> 2 atanh(tq tanh((l0 + 3m)/2)^3): each check excludes its target
  (3 of 4 edges) and each variable excludes its target (3 of 4 faces).
* Sec. 4.1 (discussion of half-cube errors): for the syndrome of a half
  stabiliser both halves are equally likely, so BP cannot choose between them
  and cannot make the error larger.  The paper states that all six qubits keep
  l > 0; flooding BP on this syndrome oscillates with the iteration count, so
  what is pinned is the symmetric outcome: the six posteriors are equal, every
  other qubit keeps l > 0, and the correction is either nothing or the whole
  stabiliser (an equivalent error with the same syndrome).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import toric3d_inputs as inp
from lattice_util import apply_map, edges_at_vertex, stabiliser, symmetry_map, vertex_edge

TREE_CHECKS = [[0, 1, 2], [2, 3, 4, 5], [5, 6], [1, 7, 8]]


def _csr(checks):
    cptr = np.cumsum([0] + [len(c) for c in checks]).astype(np.int32)
    cvar = np.array([v for c in checks for v in c], dtype=np.int32)
    return cptr, cvar


def _exact_llr(checks, nv, syn, p, q):
    num = np.zeros(nv)
    den = np.zeros(nv)
    for bits in itertools.product((0, 1), repeat=nv):
        w = 1.0
        for b in bits:
            w *= p if b else 1 - p
        for c, sc in zip(checks, syn):
            par = sum(bits[v] for v in c) % 2
            if q is None:
                if par != sc:
                    w = 0.0
                    break
            else:
                w *= q if par != sc else 1 - q
        for v in range(nv):
            if bits[v]:
                den[v] += w
            else:
                num[v] += w
    return np.log(num / den)


@pytest.mark.parametrize("meas_q", [None, 0.07])
def test_bp_exact_on_tree(meas_q):
    p = 0.1
    cptr, cvar = _csr(TREE_CHECKS)
    l0 = math.log((1 - p) / p)
    lq = math.inf if meas_q is None else math.log((1 - meas_q) / meas_q)
    for syn in itertools.product((0, 1), repeat=len(TREE_CHECKS)):
        _, llr = oracle.bp_general(cptr, cvar, np.array(syn, np.uint8), l0, lq, 12)
        exact = _exact_llr(TREE_CHECKS, 9, syn, p, meas_q)
        np.testing.assert_allclose(llr, exact, rtol=1e-9, atol=1e-9)


def test_bp_first_iteration_closed_form():
    L, p, q = 4, 0.04, 0.04
    n = 3 * L ** 3
    s = inp.random_bits(1, n, 0.1, seed=1)
    l0, lq = math.log((1 - p) / p), math.log((1 - q) / q)
    m1 = 2 * math.atanh(math.tanh(lq / 2) * math.tanh(l0 / 2) ** 3)
    msgs, llr = oracle.bp_batch(L, s, p, q, True, 1)
    sign = np.repeat(1.0 - 2.0 * s[0], 4)          # Tanner edges 4f..4f+3 belong to face f
    np.testing.assert_allclose(msgs[0], sign * m1, rtol=1e-14)
    fe, ef = oracle.incidence(L)
    want = l0 + m1 * (1.0 - 2.0 * s[0][ef]).sum(axis=1)
    np.testing.assert_allclose(llr[0], want, rtol=1e-13)


@pytest.mark.parametrize("meas", [True, False])
def test_bp_zero_syndrome_scalar_recursion(meas):
    L, p, q, iters = 3, 0.05, 0.05, 6
    n = 3 * L ** 3
    l0 = math.log((1 - p) / p)
    tq = math.tanh(math.log((1 - q) / q) / 2) if meas else 1.0
    m = None
    for _ in range(iters):
        x = l0 if m is None else l0 + 3 * m
        m = min(30.0, 2 * math.atanh(min(tq * math.tanh(x / 2) ** 3, 1 - 1e-15)))
    msgs, llr = oracle.bp_batch(L, np.zeros((1, n), np.uint8), p, q, meas, iters)
    np.testing.assert_allclose(msgs[0], m, rtol=1e-12)
    np.testing.assert_allclose(llr[0], l0 + 4 * m, rtol=1e-12)


def test_bp_continuation_from_messages():
    L, p, q = 4, 0.04, 0.04
    n = 3 * L ** 3
    s = inp.random_bits(2, n, 0.08, seed=5)
    m_full, llr_full = oracle.bp_batch(L, s, p, q, True, 7)
    m_a, _ = oracle.bp_batch(L, s, p, q, True, 3)
    m_b, llr_b = oracle.bp_batch(L, s, p, q, True, 4, m_in=m_a)
    np.testing.assert_array_equal(m_full, m_b)
    np.testing.assert_array_equal(llr_full, llr_b)


@pytest.mark.parametrize("p,meas", [(0.01, True), (0.04, True), (0.05, True), (0.04, False)])
def test_half_cube_correction_is_all_or_nothing(p, meas):
    L = 4
    V = (1, 1, 2)
    six = [vertex_edge(L, V, sp) for sp in ["+x", "-x", "+y", "-y", "+z", "-z"]]
    S = stabiliser(L, V)
    for spec in (["+x", "+y", "+z"], ["-x", "+y", "-z"]):
        e = edges_at_vertex(L, V, spec)
        s = oracle.syndrome(L, e)
        positive_seen = False
        for iters in range(1, 31):
            e2, s2, llr = oracle.bp_decode(L, e, s, p, p, meas, iters)
            assert np.ptp(llr[six]) < 1e-9
            others = np.ones(len(llr), bool)
            others[six] = False
            assert (llr[others] > 0).all()
            assert np.array_equal(e2 ^ e, 0 * S) or np.array_equal(e2 ^ e, S)
            assert np.array_equal(s2, s)
            positive_seen |= bool(llr[six[0]] > 0)
        assert positive_seen


@pytest.mark.parametrize("L", [4, 6])
@pytest.mark.parametrize("p", [0.03, 0.04, 0.051, 0.0546, 0.06])
def test_half_cube_keeps_every_llr_positive_with_30_iterations(L, p):
    """Sec. 4.1 on the half-cube error: BP cannot choose between the two halves of the
    stabiliser, every qubit of its support keeps l > 0 and nothing is corrected.  At the
    paper's BP setting (30 iterations per cycle, measurement variables, p = q) that holds
    exactly: all six posteriors of the vertex are positive and the error is unchanged."""
    V = (1, 1, 2)
    six = [vertex_edge(L, V, sp) for sp in ["+x", "-x", "+y", "-y", "+z", "-z"]]
    for spec in (["+x", "+y", "+z"], ["-x", "+y", "-z"]):
        e = edges_at_vertex(L, V, spec)
        s = oracle.syndrome(L, e)
        e2, s2, llr = oracle.bp_decode(L, e, s, p, p, True, 30)
        assert (llr[six] > 0).all() and (llr > 0).all()
        assert np.array_equal(e2, e) and np.array_equal(s2, s)


@pytest.mark.parametrize("p", [0.04, 0.0544, 0.06])
def test_half_cube_at_20_iterations_applies_the_whole_stabiliser(p):
    """Known departure from the Sec. 4.1 statement at p-BP's 20 iterations (Sec. 4.2): the
    flooding schedule oscillates on this syndrome with period 4 (the six posteriors are
    negative at iterations 2-3, 6-7, 10-11, 14-15, 18-19 and 20), so BP applies the whole
    stabiliser -- which leaves the other half of it, an equivalent error, so the paper's
    point that BP does no harm holds, but not its l > 0.  The readings of BP inside a run
    in readings.py (warm start, half-iteration counting, measurement decisions) do not
    change this: the qubits' posteriors of one decode are the same in all of them but the
    half-iteration count, which moves the decision to 10 iterations (negative too)."""
    L, V = 4, (1, 1, 2)
    six = [vertex_edge(L, V, sp) for sp in ["+x", "-x", "+y", "-y", "+z", "-z"]]
    e = edges_at_vertex(L, V, ["+x", "+y", "+z"])
    s = oracle.syndrome(L, e)
    e2, s2, llr = oracle.bp_decode(L, e, s, p, p, True, 20)
    assert (llr[six] < 0).all()
    assert np.array_equal(e2 ^ e, stabiliser(L, V)) and np.array_equal(s2, s)
    assert oracle.logical(L, e2)[0] == oracle.logical(L, e)[0]


def test_bp_posterior_commutes_with_lattice_symmetries():
    L, p = 4, 0.04
    n = 3 * L ** 3
    s = inp.random_bits(1, n, 0.06, seed=11)[0]
    m = symmetry_map(L, (2, 0, 1), (1, 0, 3))
    _, _, llr = oracle.bp_decode(L, np.zeros(n, np.uint8), s, p, p, True, 10)
    _, _, llr2 = oracle.bp_decode(L, np.zeros(n, np.uint8), apply_map(s, m), p, p, True, 10)
    out = np.zeros(n)
    out[m] = llr
    np.testing.assert_allclose(llr2, out, rtol=1e-12, atol=1e-12)


def test_bp_corrects_single_error_without_measurement_noise():
    L, p = 4, 0.02
    n = 3 * L ** 3
    for v in (0, 77, n - 1):
        e = np.zeros(n, np.uint8)
        e[v] = 1
        e2, s2, llr = oracle.bp_decode(L, e, oracle.syndrome(L, e), p, p, False, 10)
        assert e2.sum() == 0 and s2.sum() == 0 and llr[v] < 0
