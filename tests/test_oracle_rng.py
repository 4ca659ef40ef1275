"""Pins of the oracle's random-number contract.

The paper says only "random number in (0,1)" (Sec. 3.2) and nothing about how
noise is sampled, so the generator is this project's reading: Philox4x64-10
(Salmon et al., SC'11).  numpy ships an independent implementation of the same
generator, which pins every output word exactly."""
import numpy as np
import pytest

import oracle


def _numpy_block(counter, key):
    # numpy increments its 256-bit counter before producing a block
    c = sum(int(x) << (64 * i) for i, x in enumerate(counter))
    c = (c - 1) % (1 << 256)
    c_prev = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c_prev, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy():
    rng = np.random.default_rng(123)
    for _ in range(200):
        ctr = rng.integers(1, 2 ** 63, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_block(ctr, key))


def test_philox_structured_counters_match_numpy():
    # the counter shapes the library uses: (group, site, cycle, stream<<48|sweep<<8|blk)
    for group, site, cycle, word3, seed in [(1, 0, 1, 0, 0), (5, 191, 3, (2 << 48) | (7 << 8), 42),
                                            (1562, 98303, 32, (1 << 48) | 7, 2 ** 63 + 5)]:
        ctr = np.array([group, site, cycle, word3], dtype=np.uint64)
        key = np.array([seed, 0], dtype=np.uint64)
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_block(ctr, key))


def test_uniform32_bit_assembly_uses_msb_first_words():
    # U's bit (31-j) is bit `lane` of word j; word j = output j%4 of block j/4
    seed, stream, site, cycle, sweep = 9, 1, 77, 4, 0
    for sample in [64 * 3 + 0, 64 * 3 + 17, 64 * 3 + 63]:
        group, lane = sample // 64, sample % 64
        u = 0
        for blk in range(8):
            w = _numpy_block([group, site, cycle, (stream << 48) | (sweep << 8) | blk], [seed, 0])
            for i in range(4):
                j = 4 * blk + i
                u |= ((int(w[i]) >> lane) & 1) << (31 - j)
        assert oracle.uniform32(seed, stream, site, cycle, sweep, sample) == u


@pytest.mark.parametrize("p,expect", [(0.0, 0), (1.0, 1 << 32), (0.5, 1 << 31),
                                      (0.25, 1 << 30), (2.0 ** -33, 1), (2.0 ** -34, 0)])
def test_threshold_quantisation(p, expect):
    assert oracle.prob_to_threshold(p) == expect


def test_bernoulli_edges_and_frequency():
    assert all(oracle.bernoulli(0.0, 1, 0, s, 1, 0, k) == 0 for s in range(5) for k in range(70))
    assert all(oracle.bernoulli(1.0, 1, 0, s, 1, 0, k) == 1 for s in range(5) for k in range(70))
    n, p = 20000, 0.04
    hits = sum(oracle.bernoulli(p, 3, 0, i % 997, 1 + i // 997, 0, i) for i in range(n))
    sd = (n * p * (1 - p)) ** 0.5
    assert abs(hits - n * p) < 5 * sd


def test_bernoulli_is_u_less_than_threshold():
    seed = 17
    for sample in range(0, 300, 7):
        for p in (0.01, 0.04, 0.3):
            u = oracle.uniform32(seed, 0, 5, 2, 0, sample)
            assert oracle.bernoulli(p, seed, 0, 5, 2, 0, sample) == int(u < oracle.prob_to_threshold(p))


def test_coin_is_bit_of_the_sites_block_and_fair():
    """The coin of the d-edge at site r: output d of block 0 of stream 2 keyed by r."""
    seed, L = 4, 3
    for sample in (0, 1, 63, 64, 200):
        w = _numpy_block([sample // 64, 11, 3, (2 << 48) | (5 << 8)], [seed, 0])
        for d in range(3):
            assert oracle.coin(seed, L, d * L ** 3 + 11, 3, 5, sample) == (int(w[d]) >> (sample % 64)) & 1
    n = 20000
    heads = sum(oracle.coin(1, 7, i % 1029, 1, i // 1029, i) for i in range(n))
    assert abs(heads - n / 2) < 5 * (n / 4) ** 0.5


def test_streams_are_distinct():
    a = [oracle.uniform32(1, 0, 3, 1, 0, k) for k in range(64)]
    b = [oracle.uniform32(1, 1, 3, 1, 0, k) for k in range(64)]
    c = [oracle.uniform32(1, 0, 3, 2, 0, k) for k in range(64)]
    assert a != b and a != c
