"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

This module holds no decoding arithmetic: only seeded random bit patterns,
the named workload recipes, and the conversion between the oracle's
one-byte-per-bit layout ``[sample][3L^3]`` and the library's bit-sliced layout
``[3L^3][words]`` (sample ``64*w + j`` is bit ``j`` of word ``w``).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def n_bits(L: int) -> int:
    """Number of qubits (edges) and of Z checks (faces) of the L x L x L lattice."""
    return 3 * L * L * L


def words_for(n_samples: int) -> int:
    return (n_samples + 63) // 64


def random_bits(n_samples: int, n: int, density: float, seed: int) -> np.ndarray:
    """iid Bernoulli(density) bits, shape [n_samples][n], uint8."""
    rng = np.random.default_rng(seed)
    return (rng.random((n_samples, n)) < density).astype(np.uint8)


def all_patterns(n: int) -> np.ndarray:
    """Every n-bit pattern, shape [2^n][n], uint8 (sample i has bit k = (i >> k) & 1)."""
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1).astype(np.uint8)


def low_weight_patterns(n: int, max_weight: int) -> np.ndarray:
    """All patterns of weight 0..max_weight, shape [count][n], uint8."""
    from itertools import combinations
    rows = []
    for w in range(max_weight + 1):
        for c in combinations(range(n), w):
            r = np.zeros(n, dtype=np.uint8)
            r[list(c)] = 1
            rows.append(r)
    return np.stack(rows)


def pack(bits: np.ndarray) -> np.ndarray:
    """[S][n] uint8 bits -> [n][ceil(S/64)] uint64 words (tail lanes zero)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    S, n = bits.shape
    W = words_for(S)
    padded = np.zeros((W * 64, n), dtype=np.uint8)
    padded[:S] = bits
    by = np.packbits(padded.T.reshape(n, W, 64), axis=2, bitorder="little")  # [n][W][8]
    return np.ascontiguousarray(by).view(np.uint64).reshape(n, W)


def unpack(words: np.ndarray, n_samples: int) -> np.ndarray:
    """[n][W] uint64 words -> [n_samples][n] uint8 bits."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    n, W = words.shape
    by = words.view(np.uint8).reshape(n, W, 8)
    bits = np.unpackbits(by, axis=2, bitorder="little").reshape(n, W * 64)
    return np.ascontiguousarray(bits[:, :n_samples].T)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: lattice size, noise, decoder and batch."""

    name: str
    L: int
    p: float
    q: float
    T: int
    n_samples: int
    seed: int
    decoder: str            # "flip" | "pflip" | "bp_pflip" | "bp"
    schedule: str = ""
    n_apply: int = 0            # rule applications per cycle (schedule string cycled)
    bp_iters: int = 0
    bp_meas_nodes: bool = True
    perfect_round: bool = False
    perfect_max_sweeps: int = 0
    extra_L: tuple = ()         # further lattice sizes decoded in the same launches

    @property
    def sizes(self):
        return (self.L,) + tuple(self.extra_L)


# Workload recipes (phenomenological noise with p = q throughout, as in the
# paper's simulations; every input is drawn from the seeded Philox streams).
WORKLOADS = {
    # plain flip, L=4, T=4 + perfect round, up to 32 sweeps, 10^4 samples
    "flip_L4": Workload("flip_L4", 4, 0.01, 0.01, 4, 10_000, 0, "flip", "F", 32,
                        perfect_round=True, perfect_max_sweeps=32),
    # p-flip with the Sec. 3.2 example schedule FFPFF, T=L, 10^6 samples per point
    "pflip_L8": Workload("pflip_L8", 8, 0.03, 0.03, 8, 1_000_000, 1000, "pflip", "FFPFF", 5),
    "pflip_L16": Workload("pflip_L16", 16, 0.03, 0.03, 16, 1_000_000, 1000, "pflip", "FFPFF", 5),
    "pflip_L32": Workload("pflip_L32", 32, 0.04, 0.04, 32, 100_000, 17, "pflip", "FFPFF", 5),
    # BP (16 FP32 iterations) + 32 applications cycling PFFPFF, T=L
    "bp_pflip_L16": Workload("bp_pflip_L16", 16, 0.04, 0.04, 16, 100_000, 7, "bp_pflip",
                             "PFFPFF", 32, bp_iters=16),
    # L=16 and L=24 mixed in one persistent launch per step, 10^5 samples each
    "bp_pflip_L16_L24": Workload("bp_pflip_L16_L24", 16, 0.04, 0.04, 16, 100_000, 7, "bp_pflip",
                                 "PFFPFF", 32, bp_iters=16, extra_L=(24,)),
    # throughput point: L=32, p=q=4%, T=L, 10^5 samples, BP16 + 32 x PFFPFF
    "bp_pflip_L32": Workload("bp_pflip_L32", 32, 0.04, 0.04, 32, 100_000, 11, "bp_pflip",
                             "PFFPFF", 32, bp_iters=16),
    "bp_pflip_L48": Workload("bp_pflip_L48", 48, 0.04, 0.04, 48, 100_000, 13, "bp_pflip",
                             "PFFPFF", 32, bp_iters=16),
}


# ---------------------------------------------------------------- other LDPC codes
# Code structure only (parity-check matrices as CSR lists), for the generic
# Tanner-graph decoders: seeded random biregular classical codes and their
# hypergraph product (Tillich-Zemor), whose Z checks are a quantum LDPC code
# with the same kind of local, low-degree Tanner graph as the toric code.

def random_biregular(n: int, m: int, dv: int, dc: int, seed: int) -> np.ndarray:
    """A classical parity-check matrix as the [m][dc] bit indices of its rows: column
    weight dv, row weight dc (n dv = m dc), from the configuration model; a row that
    repeats a bit swaps that entry with a random entry of another row until every row
    is simple."""
    assert n * dv == m * dc, "n dv must equal m dc"
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), dv)
    rng.shuffle(rows)
    rows = rows.reshape(m, dc)
    for _ in range(100 * m * dc):
        bad = [r for r in range(m) if len(set(rows[r].tolist())) < dc]
        if not bad:
            return rows
        r = bad[0]
        vals, counts = np.unique(rows[r], return_counts=True)
        k = int(np.nonzero(rows[r] == vals[counts > 1][0])[0][0])
        r2, k2 = int(rng.integers(m)), int(rng.integers(dc))
        rows[r, k], rows[r2, k2] = rows[r2, k2], rows[r, k]
    raise RuntimeError("no simple biregular graph found")


def cyclic_repetition(L: int) -> np.ndarray:
    """Rows {i, i+1 mod L} of the length-L cyclic repetition code, [L][2]."""
    return np.stack([np.arange(L), (np.arange(L) + 1) % L], axis=1)


def hypergraph_product(rows1: np.ndarray, n1: int, rows2: np.ndarray, n2: int):
    """Check lists (one list of qubit indices per check) of the hypergraph product of
    the classical codes with rows rows1 (m1 checks on n1 bits) and rows2 (m2 on n2):
    qubits (a, b) -> a n2 + b for the n1 n2 bit pairs, then n1 n2 + i m2 + j for the
    m1 m2 check pairs;  X check (i, b) = {(a, b) : a in row i of code 1} +
    {(i, j) : b in row j of code 2};  Z check (a, j) = {(a, b) : b in row j of code 2}
    + {(i, j) : a in row i of code 1}, i.e. HX = [H1 x I | I x H2^T],
    HZ = [I x H2 | H1^T x I]."""
    m1, m2 = len(rows1), len(rows2)
    rows_of_bit1 = [[] for _ in range(n1)]
    for i, r in enumerate(rows1):
        for a in r:
            rows_of_bit1[int(a)].append(i)
    rows_of_bit2 = [[] for _ in range(n2)]
    for j, r in enumerate(rows2):
        for b in r:
            rows_of_bit2[int(b)].append(j)
    base = n1 * n2
    X = [[int(a) * n2 + b for a in rows1[i]] + [base + i * m2 + j for j in rows_of_bit2[b]]
         for i in range(m1) for b in range(n2)]
    Z = [[a * n2 + int(b) for b in rows2[j]] + [base + i * m2 + j for i in rows_of_bit1[a]]
         for a in range(n1) for j in range(m2)]
    return X, Z, n1 * n2 + m1 * m2


def csr(check_lists):
    """Check lists as CSR (cptr int32 [m+1], cvar int32 [nnz], each row sorted)."""
    cptr = np.zeros(len(check_lists) + 1, dtype=np.int64)
    cptr[1:] = np.cumsum([len(c) for c in check_lists])
    cvar = np.concatenate([np.sort(np.asarray(c, dtype=np.int64)) for c in check_lists])
    return cptr.astype(np.int32), cvar.astype(np.int32)


def hgp_workload(n_classical: int, seed: int):
    """Z checks of the hypergraph product of two seeded (3, 4)-biregular classical codes
    with n_classical bits and 3 n_classical / 4 checks each: n^2 + (3n/4)^2 qubits,
    3n^2/4 checks of weight 7, qubit degree 3 or 4.  Returns (cptr, cvar, n_qubits)."""
    m = 3 * n_classical // 4
    r1 = random_biregular(n_classical, m, 3, 4, seed)
    r2 = random_biregular(n_classical, m, 3, 4, seed + 1)
    _, Z, n = hypergraph_product(r1, n_classical, r2, n_classical)
    cptr, cvar = csr(Z)
    return cptr, cvar, n
