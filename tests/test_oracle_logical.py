"""Pins of the oracle's logical readout (Sec. 3.1 and its footnote, Fig. 2
caption, App. A.2).

For axis d the logical Z operators are the L^2 disjoint straight lines of
d-edges; a membrane of L^2 parallel d-edges (a logical X, Sec. 2) crosses
every d-line once, so it flips every line parity and the majority vote reports
a logical X error on qubit d only.  Stabilisers commute with every logical Z,
so they leave all parities unchanged.  On a codeword (zero syndrome) the line
parities along an axis are unanimous.  The paper gives no tie rule; a tie
(exactly half of the lines odd) counts as a failure here."""
import numpy as np
import pytest

import oracle
import toric3d_inputs as inp
from lattice_util import idx, membrane, stabiliser


@pytest.mark.parametrize("L", [3, 4, 5])
def test_membrane_flips_exactly_its_axis(L):
    for d in range(3):
        for c in (0, L - 1):
            m, counts = oracle.logical(L, membrane(L, d, c))
            assert m == 1 << d
            assert counts[d] == L * L and counts.sum() == L * L


@pytest.mark.parametrize("L", [3, 4])
def test_stabilisers_leave_parities_unchanged(L):
    e = inp.random_bits(1, 3 * L ** 3, 0.1, seed=L)[0]
    _, c0 = oracle.logical(L, e)
    rng = np.random.default_rng(0)
    for _ in range(10):
        v = tuple(int(x) for x in rng.integers(0, L, 3))
        e = e ^ stabiliser(L, v)
        _, c = oracle.logical(L, e)
        assert np.array_equal(c, c0)


@pytest.mark.parametrize("L", [3, 4])
def test_codewords_have_unanimous_lines(L):
    rng = np.random.default_rng(L)
    for _ in range(20):
        e = np.zeros(3 * L ** 3, np.uint8)
        want = 0
        for d in range(3):
            if rng.random() < 0.5:
                e ^= membrane(L, d, int(rng.integers(L)))
                want ^= 1 << d
        for _ in range(int(rng.integers(0, 30))):
            e ^= stabiliser(L, tuple(int(x) for x in rng.integers(0, L, 3)))
        assert oracle.syndrome(L, e).sum() == 0
        m, counts = oracle.logical(L, e)
        assert m == want
        assert all(c in (0, L * L) for c in counts)


def test_tie_counts_as_failure():
    L = 4
    e = np.zeros(3 * L ** 3, np.uint8)
    # one x-edge on each of L^2/2 distinct x-lines (line = fixed (y, z))
    lines = [(y, z) for y in range(L) for z in range(L)][: L * L // 2]
    for y, z in lines:
        e[idx(L, 0, 1, y, z)] = 1
    m, counts = oracle.logical(L, e)
    assert counts[0] == L * L // 2 and m == 1
    e[idx(L, 0, 1, *lines[0])] = 0
    m, counts = oracle.logical(L, e)
    assert counts[0] == L * L // 2 - 1 and m == 0


def test_odd_lattice_majority_threshold():
    L = 3
    lines = [(y, z) for y in range(L) for z in range(L)]
    for k, want in [(4, 0), (5, 1)]:
        e = np.zeros(3 * L ** 3, np.uint8)
        for (y, z) in lines[:k]:
            e[idx(L, 0, (y + z) % L, y, z)] = 1
        m, counts = oracle.logical(L, e)
        assert counts[0] == k and m == want
