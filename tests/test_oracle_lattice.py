"""Pins of the oracle's lattice and syndrome map against Sec. 2 of the paper.

Sec. 2 fixes the code as [[3L^3, 3, L]] with every Z check on 4 qubits and
every qubit in 4 Z checks; the vertex (X) stabilisers have rank L^3 - 1, so the
face-check matrix H must have GF(2) rank 3L^3 - 3 - (L^3 - 1) = 2L^3 - 2.  X
errors give looplike syndromes: every cube sees an even number of violated
faces.  A stabiliser and a minimum-weight logical X (a membrane of L^2 parallel
edges) have zero syndrome."""
import numpy as np
import pytest

import oracle
import toric3d_inputs as inp
from lattice_util import (cube_faces, gf2_rank, membrane, stabiliser, symmetry_map, apply_map)


def _check_matrix(L):
    n = 3 * L ** 3
    H = np.zeros((n, n), dtype=np.uint8)
    for v in range(n):
        e = np.zeros(n, dtype=np.uint8)
        e[v] = 1
        H[:, v] = oracle.syndrome(L, e)
    return H


@pytest.mark.parametrize("L", [2, 3, 4])
def test_rank_and_weights(L):
    H = _check_matrix(L)
    assert (H.sum(axis=0) == 4).all(), "every qubit must be in exactly 4 Z checks"
    assert (H.sum(axis=1) == 4).all(), "every Z check must touch exactly 4 qubits"
    assert gf2_rank(H) == 2 * L ** 3 - 2


@pytest.mark.parametrize("L", [3, 5])
def test_single_edge_lights_four_faces(L):
    n = 3 * L ** 3
    for v in range(0, n, 7):
        e = np.zeros(n, dtype=np.uint8)
        e[v] = 1
        assert oracle.syndrome(L, e).sum() == 4


@pytest.mark.parametrize("L", [3, 4, 6])
def test_noiseless_syndrome_is_closed_on_every_cube(L):
    e = inp.random_bits(1, 3 * L ** 3, 0.2, seed=L)[0]
    s = oracle.syndrome(L, e)
    for x in range(L):
        for y in range(L):
            for z in range(L):
                assert s[cube_faces(L, (x, y, z))].sum() % 2 == 0


@pytest.mark.parametrize("L", [2, 3, 4])
def test_stabilisers_and_membranes_have_zero_syndrome(L):
    for v in [(0, 0, 0), (1, L - 1, 0), (L - 1, L - 1, L - 1)]:
        assert oracle.syndrome(L, stabiliser(L, v)).sum() == 0
    for d in range(3):
        for c in range(L):
            m = membrane(L, d, c)
            assert m.sum() == L * L
            assert oracle.syndrome(L, m).sum() == 0


def test_face_edges_geometry():
    L = 5
    # face with normal z at (1,2,3) is spanned by x and y
    f = ((2 * L + 3) * L + 2) * L + 1
    got = sorted(oracle.face_edges(L, f).tolist())
    want = sorted([((0 * L + 3) * L + 2) * L + 1, ((0 * L + 3) * L + 3) * L + 1,
                   ((1 * L + 3) * L + 2) * L + 1, ((1 * L + 3) * L + 2) * L + 2])
    assert got == want


@pytest.mark.parametrize("perm", [(0, 1, 2), (1, 2, 0), (2, 0, 1), (1, 0, 2), (0, 2, 1), (2, 1, 0)])
def test_syndrome_commutes_with_lattice_symmetries(perm):
    L = 4
    e = inp.random_bits(1, 3 * L ** 3, 0.15, seed=7)[0]
    m = symmetry_map(L, perm, (1, 3, 2))
    assert np.array_equal(oracle.syndrome(L, apply_map(e, m)), apply_map(oracle.syndrome(L, e), m))


def test_incidence_tables_are_inverse():
    L = 3
    fe, ef = oracle.incidence(L)
    for f in range(3 * L ** 3):
        for v in fe[f]:
            assert f in ef[v]
    assert all(len(set(row)) == 4 for row in ef)
