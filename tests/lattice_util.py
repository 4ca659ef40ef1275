"""Test-side helpers: coordinates of the public index layout, lattice symmetries
and small named error patterns from the paper's worked examples.

Layout (the library's and the oracle's interface):
    edge (d, x, y, z) -> ((d*L + z)*L + y)*L + x
    face (n, x, y, z) -> ((n*L + z)*L + y)*L + x
"""
from __future__ import annotations

import numpy as np


def idx(L, d, x, y, z):
    return ((d * L + z % L) * L + y % L) * L + x % L


def coords(L):
    """(kind, x, y, z) arrays for every index 0..3L^3-1."""
    i = np.arange(3 * L ** 3)
    return i // L ** 3, i % L, (i // L) % L, (i // (L * L)) % L


def symmetry_map(L, perm, shift):
    """Index map of the lattice symmetry 'relabel axis i as perm[i], then translate'.

    Valid for edges and faces alike (the kind index is an axis label in both)."""
    k, x, y, z = coords(L)
    r = np.stack([x, y, z])
    r2 = np.empty_like(r)
    for i in range(3):
        r2[perm[i]] = (r[i] + shift[perm[i]]) % L
    k2 = np.asarray(perm)[k]
    return ((k2 * L + r2[2]) * L + r2[1]) * L + r2[0]


def apply_map(bits, m):
    out = np.zeros_like(bits)
    out[..., m] = bits
    return out


AX = {"x": 0, "y": 1, "z": 2}


def vertex_edge(L, v, spec):
    """Edge at vertex v named '+x', '-y', ...: '+a' leaves v along a, '-a' arrives at v."""
    sign, a = spec[0], AX[spec[1]]
    r = list(v)
    if sign == "-":
        r[a] -= 1
    return idx(L, a, *r)


def edges_at_vertex(L, v, specs):
    e = np.zeros(3 * L ** 3, dtype=np.uint8)
    for sp in specs:
        e[vertex_edge(L, v, sp)] ^= 1
    return e


def stabiliser(L, v):
    """X stabiliser at vertex v: its six edges."""
    return edges_at_vertex(L, v, ["+x", "-x", "+y", "-y", "+z", "-z"])


def membrane(L, d, c):
    """All L^2 edges of direction d whose d-coordinate is c (a logical X)."""
    e = np.zeros(3 * L ** 3, dtype=np.uint8)
    for u in range(L):
        for w in range(L):
            r = [0, 0, 0]
            r[d] = c
            others = [a for a in range(3) if a != d]
            r[others[0]], r[others[1]] = u, w
            e[idx(L, d, *r)] = 1
    return e


def cube_faces(L, r):
    """The six faces bounding the unit cube whose lowest corner is r."""
    out = []
    for n in range(3):
        out.append(idx(L, n, *r))
        r2 = list(r)
        r2[n] += 1
        out.append(idx(L, n, *r2))
    return out


def gf2_rank(rows):
    """Rank over GF(2) of a 0/1 matrix given as a 2-D array."""
    ints = [int("".join("1" if b else "0" for b in row), 2) for row in np.asarray(rows)]
    rank = 0
    pivots = {}
    for v in ints:
        while v:
            top = v.bit_length() - 1
            if top in pivots:
                v ^= pivots[top]
            else:
                pivots[top] = v
                rank += 1
                break
    return rank
