"""Pins of the oracle's flip and p-flip against the worked examples of Sec. 3.

* A single X error is removed by one parallel application (Sec. 3.1: every
  qubit of it sees 4 unsatisfied checks, its neighbours at most 1).
* Fig. 3(a): three of the six qubits of an X stabiliser (one per axis at a
  vertex) -- each sees 2 satisfied and 2 unsatisfied checks, so flip is stuck.
* Fig. 3(b): four parallel qubits on a 2x2 plaquette -- also stuck.
* Sec. 3.2: for the half-cube the qubits with 2 satisfied / 2 unsatisfied
  checks are exactly the six qubits of that stabiliser, so p-flip flips a
  subset of them chosen by the coins.
* Sec. 3.2: two errors on opposite faces of a stabiliser cube are removed by
  a single application of flip.
* Fig. 5: the parallel rule maps a three-qubit error to a rotated copy and
  back (period 2); the sequential rule of Sec. 3.1 corrects it.
* Fig. 4(a): a fourth error on the half-cube's stabiliser makes it
  correctable.
"""
import numpy as np
import pytest

import oracle
import toric3d_inputs as inp
from lattice_util import (apply_map, edges_at_vertex, stabiliser, symmetry_map, vertex_edge)

L = 4
V = (1, 2, 1)
HALF_CUBES = [[sx + "x", sy + "y", sz + "z"] for sx in "+-" for sy in "+-" for sz in "+-"]


def _flip(e):
    return oracle.flip_once(L, e, oracle.syndrome(L, e))


@pytest.mark.parametrize("Lx", [3, 4])
def test_single_error_removed_in_one_application(Lx):
    n = 3 * Lx ** 3
    for v in range(n):
        e = np.zeros(n, dtype=np.uint8)
        e[v] = 1
        e2, s2 = oracle.flip_once(Lx, e, oracle.syndrome(Lx, e))
        assert e2.sum() == 0 and s2.sum() == 0


@pytest.mark.parametrize("spec", HALF_CUBES)
def test_half_cube_is_fixed_point_of_flip(spec):
    e = edges_at_vertex(L, V, spec)
    s = oracle.syndrome(L, e)
    assert s.sum() == 6
    e2, s2 = oracle.flip_once(L, e, s)
    assert np.array_equal(e2, e) and np.array_equal(s2, s)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_planar_plaquette_is_fixed_point_of_flip(d):
    from lattice_util import idx
    e = np.zeros(3 * L ** 3, dtype=np.uint8)
    a, b = [x for x in range(3) if x != d]
    for da in (0, 1):
        for db in (0, 1):
            r = [1, 1, 1]
            r[a] += da
            r[b] += db
            e[idx(L, d, *r)] = 1
    s = oracle.syndrome(L, e)
    assert s.sum() == 8
    e2, s2 = oracle.flip_once(L, e, s)
    assert np.array_equal(e2, e) and np.array_equal(s2, s)


@pytest.mark.parametrize("spec", HALF_CUBES[:3])
def test_pflip_on_half_cube_flips_coin_chosen_vertex_edges(spec):
    e = edges_at_vertex(L, V, spec)
    s = oracle.syndrome(L, e)
    six = [vertex_edge(L, V, sp) for sp in ["+x", "-x", "+y", "-y", "+z", "-z"]]
    seen = set()
    for sample in range(40):
        e2, _ = oracle.pflip_once(L, e, s, seed=5, sample=sample, cycle=1, sweep=2)
        flipped = set(np.nonzero(e2 ^ e)[0].tolist())
        want = {v for v in six if oracle.coin(5, L, v, 1, 2, sample)}
        assert flipped == want
        seen |= flipped
    assert seen == set(six)


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_opposite_face_pair_removed_by_one_flip(axis):
    e = edges_at_vertex(L, V, ["+" + axis, "-" + axis])
    e2, s2 = _flip(e)
    assert e2.sum() == 0 and s2.sum() == 0


def test_opposite_face_pair_under_pflip_only_touches_the_cube():
    e = edges_at_vertex(L, V, ["+z", "-z"])
    s = oracle.syndrome(L, e)
    cube = {vertex_edge(L, V, sp) for sp in ["+x", "-x", "+y", "-y"]}
    for sample in range(20):
        e2, _ = oracle.pflip_once(L, e, s, seed=1, sample=sample, cycle=1, sweep=0)
        assert set(np.nonzero(e2)[0].tolist()) == {v for v in cube if oracle.coin(1, L, v, 1, 0, sample)}


def test_fig5_pair_oscillates_under_parallel_flip():
    a = edges_at_vertex(L, V, ["+z", "-z", "+y"])
    b = edges_at_vertex(L, V, ["+x", "-x", "+y"])
    a1, _ = _flip(a)
    assert np.array_equal(a1, b)
    a2, _ = _flip(a1)
    assert np.array_equal(a2, a)


def test_fig5_pair_is_corrected_by_sequential_flip():
    a = edges_at_vertex(L, V, ["+z", "-z", "+y"])
    e2, s2, k = oracle.flip_sequential(L, a, oracle.syndrome(L, a))
    assert k > 0 and s2.sum() == 0
    m, _ = oracle.logical(L, e2)
    assert m == 0


@pytest.mark.parametrize("extra", ["-x", "-y", "-z"])
def test_fig4a_fourth_error_makes_half_cube_correctable(extra):
    e = edges_at_vertex(L, V, ["+x", "+y", "+z", extra])
    s = oracle.syndrome(L, e)
    for _ in range(10):
        if s.sum() == 0:
            break
        e, s = oracle.flip_once(L, e, s)
    assert s.sum() == 0
    m, _ = oracle.logical(L, e)
    assert m == 0


def test_flip_commutes_with_lattice_symmetries():
    e = inp.random_bits(1, 3 * L ** 3, 0.08, seed=3)[0]
    s = oracle.syndrome(L, e) ^ inp.random_bits(1, 3 * L ** 3, 0.05, seed=4)[0]
    for perm, shift in [((1, 2, 0), (0, 1, 3)), ((2, 1, 0), (2, 2, 1))]:
        m = symmetry_map(L, perm, shift)
        e1, s1 = oracle.flip_once(L, e, s)
        e2, s2 = oracle.flip_once(L, apply_map(e, m), apply_map(s, m))
        assert np.array_equal(e2, apply_map(e1, m)) and np.array_equal(s2, apply_map(s1, m))


def test_flip_keeps_syndrome_consistent_with_error():
    # s ^= H f: after any number of applications s = H e xor (initial measurement error)
    n = 3 * L ** 3
    e = inp.random_bits(1, n, 0.05, seed=8)[0]
    meas = inp.random_bits(1, n, 0.03, seed=9)[0]
    s = oracle.syndrome(L, e) ^ meas
    for k in range(6):
        if k % 3 == 2:
            e, s = oracle.pflip_once(L, e, s, 2, 0, 1, k)
        else:
            e, s = oracle.flip_once(L, e, s)
        assert np.array_equal(s, oracle.syndrome(L, e) ^ meas)


def test_stabiliser_times_error_has_same_flip_dynamics_on_syndrome():
    # the decoder sees only the syndrome, so e and e*S evolve to results differing by S
    e = inp.random_bits(1, 3 * L ** 3, 0.05, seed=12)[0]
    S = stabiliser(L, (2, 0, 3))
    s = oracle.syndrome(L, e)
    e1, s1 = oracle.flip_once(L, e, s)
    e2, s2 = oracle.flip_once(L, e ^ S, s)
    assert np.array_equal(e1 ^ e2, S) and np.array_equal(s1, s2)
