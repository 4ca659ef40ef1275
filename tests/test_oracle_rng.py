"""Pins of the oracle's random-number contract.

The paper says only "random number in (0,1)" (Sec. 3.2) and nothing about how
noise is sampled, so the generator is this project's reading: Philox4x32-10
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11).  Two pins independent of the oracle: the generator's published
known-answer vectors (the philox4x32 10-round entries of the Random123
distribution's kat_vectors), and Triton's own implementation of the same
generator (triton.language.random.philox_impl, run by Triton's CPU
interpreter) on random counters and keys and on the counter shapes the
library uses."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

# Random123 kat_vectors, philox4x32 with 10 rounds: (counter, key, output)
KAT = [
    ([0x00000000, 0x00000000, 0x00000000, 0x00000000], [0x00000000, 0x00000000],
     [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff], [0xffffffff, 0xffffffff],
     [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox4x32(ctr, key).tolist() == out


_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
from triton.language.random import philox_impl

@triton.jit
def k(ctr_ptr, key_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(ctr_ptr + 4 * i); c1 = tl.load(ctr_ptr + 4 * i + 1)
    c2 = tl.load(ctr_ptr + 4 * i + 2); c3 = tl.load(ctr_ptr + 4 * i + 3)
    k0 = tl.load(key_ptr + 2 * i); k1 = tl.load(key_ptr + 2 * i + 1)
    o0, o1, o2, o3 = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out_ptr + 4 * i, o0); tl.store(out_ptr + 4 * i + 1, o1)
    tl.store(out_ptr + 4 * i + 2, o2); tl.store(out_ptr + 4 * i + 3, o3)

data = json.loads(sys.stdin.read())
n = len(data["key"]) // 2
N = 1
while N < n:
    N *= 2
ctr = torch.zeros(4 * N, dtype=torch.int64)
ctr[:4 * n] = torch.tensor(data["ctr"], dtype=torch.int64)
key = torch.zeros(2 * N, dtype=torch.int64)
key[:2 * n] = torch.tensor(data["key"], dtype=torch.int64)
out = torch.zeros(4 * N, dtype=torch.uint32)
k[(1,)](ctr.to(torch.uint32), key.to(torch.uint32), out, N)
print(json.dumps([int(x) & 0xffffffff for x in out[:4 * n].tolist()]))
"""


def _triton_blocks(ctrs, keys):
    """Philox4x32-10 blocks from Triton's implementation, in a separate process (the
    interpreter mode is process-wide)."""
    pytest.importorskip("triton")
    import json
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], capture_output=True, text=True, timeout=600,
                       input=json.dumps({"ctr": [int(x) for c in ctrs for x in c],
                                         "key": [int(x) for k in keys for x in k]}))
    if r.returncode != 0:
        pytest.skip("Triton's CPU interpreter is unavailable: " + r.stderr.strip().splitlines()[-1][:200])
    flat = json.loads(r.stdout.strip().splitlines()[-1])
    return [flat[4 * i:4 * i + 4] for i in range(len(ctrs))]


def test_philox_matches_triton():
    rng = np.random.default_rng(123)
    ctrs = rng.integers(0, 2 ** 32, (60, 4), dtype=np.uint64)
    keys = rng.integers(0, 2 ** 32, (60, 2), dtype=np.uint64)
    # the counter shapes the library uses: (group, site, cycle, stream<<30|sweep<<8|block), key (seed lo, seed hi)
    shaped = [([1, 0, 1, 0], [0, 0]), ([5, 191, 3, (2 << 30) | (7 << 8)], [42, 0]),
              ([1562, 98303, 32, (1 << 30) | 15], [5, 1 << 31]), ([15624, 331775, 1000, (2 << 30) | (63 << 8) | 1],
                                                                  [0xdeadbeef, 0x12345678])]
    ctrs = [list(c) for c in ctrs] + [c for c, _ in shaped]
    keys = [list(k) for k in keys] + [k for _, k in shaped]
    want = _triton_blocks(ctrs, keys)
    for c, k, w in zip(ctrs, keys, want):
        assert oracle.philox4x32(c, k).tolist() == w


def _word(seed, stream, site, cycle, sweep, group, i):
    """Word i of a stream position, assembled from single blocks as the contract states."""
    out = oracle.philox4x32([group % 2 ** 32, site, cycle, (stream << 30) | (sweep << 8) | (i // 2)],
                            [seed % 2 ** 32, seed >> 32])
    j = 2 * (i % 2)
    return int(out[j]) | (int(out[j + 1]) << 32)


def _high6(seed, stream, site, cycle, sweep, group):
    """The six high bits of U for the 64 lanes of a group, from stream words 0..5 (bit 5-j of
    lane l is bit l of word j)."""
    words = [_word(seed, stream, site, cycle, sweep, group, j) for j in range(6)]
    return [sum(((words[j] >> l) & 1) << (5 - j) for j in range(6)) for l in range(64)]


@pytest.mark.parametrize("m", [1, 5, 32, 63])
def test_bernoulli_is_the_six_bit_comparison_when_p_is_a_multiple_of_one_64th(m):
    # P = m 2^26 has zero low bits, so U < P iff U's six high bits are below m
    seed, stream, site, cycle = 7 + (1 << 33), 1, 913, 6
    for group in (0, 5, 1000):
        h = _high6(seed, stream, site, cycle, 0, group)
        got = [oracle.bernoulli(m / 64, seed, stream, site, cycle, 0, 64 * group + l) for l in range(64)]
        assert got == [int(x < m) for x in h]


def test_bernoulli_tied_lanes_take_block_outputs_in_lane_order():
    # groups with at least five lanes whose six high bits tie P's (block 4 serves the fifth);
    # three thresholds with the same high bits and low parts 1/4, 1/2, 3/4 read three bits of
    # each tied lane's tail
    seed, stream, site, cycle, ph = 3, 0, 41, 2, 19
    ps = [(ph + f) / 64 for f in (0.25, 0.5, 0.75)]
    found = 0
    for group in range(40000):
        h = _high6(seed, stream, site, cycle, 0, group)
        tied = [l for l in range(64) if h[l] == ph]
        if len(tied) < 5:
            continue
        found += 1
        for p in ps:
            P = oracle.prob_to_threshold(p)
            assert P >> 26 == ph
            pl = P & ((1 << 26) - 1)
            for k, lane in enumerate(tied):
                out = oracle.philox4x32([group, site, cycle, (stream << 30) | (3 + k // 4)], [seed, 0])
                want = int((int(out[k % 4]) >> 6) < pl)
                assert oracle.bernoulli(p, seed, stream, site, cycle, 0, 64 * group + lane) == want, (group, k)
            for lane in set(range(64)) - set(tied):
                assert oracle.bernoulli(p, seed, stream, site, cycle, 0, 64 * group + lane) == int(h[lane] < ph)
        if found == 3:
            break
    assert found == 3


@pytest.mark.parametrize("p", [0.004, 0.04, 0.3, 0.5 + 2.0 ** -30])
def test_bernoulli_frequency(p):
    # p = 0.004 < 1/64: every event comes from a tied lane's 26-bit tail
    n = 64 * 2000
    hits = sum(oracle.bernoulli_count(p, 11, 0, site, 3, 0, 0, n) for site in range(4))
    N, q = 4 * n, oracle.prob_to_threshold(p) / 2 ** 32
    assert abs(hits - N * q) < 5 * (N * q * (1 - q)) ** 0.5


def test_bernoulli_lanes_of_a_word_are_independent():
    # words with two or more events follow Binomial(64, p); tied lanes that shared a tail
    # value would cluster their events (about 2.5x as many such words at p = 0.004)
    p, n = 0.004, 20000
    q = oracle.prob_to_threshold(p) / 2 ** 32
    multi = sum(oracle.bernoulli_count(p, 5, 1, 77, 9, 0, 64 * g, 64) >= 2 for g in range(n))
    f = 1 - (1 - q) ** 64 - 64 * q * (1 - q) ** 63
    assert abs(multi - n * f) < 5 * (n * f * (1 - f)) ** 0.5


def test_bernoulli_is_monotone_in_p():
    # U < P1 implies U < P2 for P1 <= P2, the tied lanes' tails included
    ps = [0.001, 0.004, 0.0156, 0.0157, 0.04, 0.0401, 0.3, 0.7]
    for sample in range(0, 64 * 40, 3):
        ev = [oracle.bernoulli(p, 21, 0, 300, 4, 0, sample) for p in ps]
        assert ev == sorted(ev), sample


def test_bernoulli_edges():
    assert all(oracle.bernoulli(0.0, 1, 0, s, 1, 0, k) == 0 for s in range(5) for k in range(70))
    assert all(oracle.bernoulli(1.0, 1, 0, s, 1, 0, k) == 1 for s in range(5) for k in range(70))


def test_coin_is_bit_of_the_sites_words_and_fair():
    """The coin of the d-edge at site r: word d of stream 2 keyed by r."""
    seed, L = 4, 3
    for sample in (0, 1, 63, 64, 200):
        for d in range(3):
            w = _word(seed, 2, 11, 3, 5, sample // 64, d)
            assert oracle.coin(seed, L, d * L ** 3 + 11, 3, 5, sample) == (w >> (sample % 64)) & 1
    n = 20000
    heads = sum(oracle.coin(1, 7, i % 1029, 1, i // 1029, i) for i in range(n))
    assert abs(heads - n / 2) < 5 * (n / 4) ** 0.5


def test_streams_are_distinct():
    a = [oracle.bernoulli(0.5, 1, 0, 3, 1, 0, k) for k in range(64)]
    b = [oracle.bernoulli(0.5, 1, 1, 3, 1, 0, k) for k in range(64)]
    c = [oracle.bernoulli(0.5, 1, 0, 3, 2, 0, k) for k in range(64)]
    assert a != b and a != c
