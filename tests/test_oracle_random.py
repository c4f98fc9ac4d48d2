"""Pins of the oracle's random draws: Philox4x32-10 word streams and Lemire
bounded integers, checked by their statistical properties and against the
independent Philox of the input generator."""
import numpy as np
from scipy import stats

import oracle
from paper_2202_00517_gb300 import datagen


def test_words_uniform_bytes():
    w = oracle.stream_words(12345, 7, 0, 0, 200_000)
    for shift in (0, 8, 16, 24):
        counts = np.bincount((w >> shift) & 0xFF, minlength=256)
        assert stats.chisquare(counts).pvalue > 1e-4


def test_words_bit_balance():
    w = oracle.stream_words(1, 0, 0, 0, 100_000)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(0)
    assert np.all(np.abs(bits - 0.5) < 0.01)


def test_avalanche_on_counter_bit():
    base = np.array([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], dtype=np.uint32)
    key = np.array([0xA4093822, 0x299F31D0], dtype=np.uint32)
    out0 = oracle.philox4x32_10(base, key)
    flips = []
    for word in range(4):
        for bit in range(32):
            c = base.copy()
            c[word] ^= np.uint32(1 << bit)
            d = oracle.philox4x32_10(c, key) ^ out0
            flips.append(sum(bin(int(v)).count("1") for v in d))
    flips = np.array(flips)
    assert 58 < flips.mean() < 70
    assert flips.min() > 30


def test_streams_differ_by_seed_and_counter():
    a = oracle.stream_words(5, 1, 2, 0, 64)
    assert not np.array_equal(a, oracle.stream_words(6, 1, 2, 0, 64))
    assert not np.array_equal(a, oracle.stream_words(5, 2, 2, 0, 64))
    assert not np.array_equal(a, oracle.stream_words(5, 1, 3, 0, 64))
    assert not np.array_equal(a, oracle.stream_words(5, 1, 2, 1, 64))
    # block j+1 follows block j: words 4..7 are the block-1 output
    ctr = np.array([1, 2, 0, 1], dtype=np.uint32)
    key = np.array([5, 0], dtype=np.uint32)
    assert np.array_equal(a[4:8], oracle.philox4x32_10(ctr, key))


def test_matches_input_generator_philox():
    seed = (0xDEADBEEF << 32) | 0x12345678
    c0 = np.arange(0, 50, dtype=np.uint64)
    for blk in range(3):
        ref = datagen._philox_blocks(c0, 0, 2, blk, seed)
        for i in (0, 17, 49):
            got = oracle.stream_words(seed, int(c0[i]), 0, 2, 12)[4 * blk:4 * blk + 4]
            assert np.array_equal(got, ref[i])


def test_bounded_small_ranges():
    assert np.all(oracle.bounded_draws(3, 0, 0, 0, 1, 1000) == 0)
    for N in (2, 7, 10, 1999):
        d = oracle.bounded_draws(99, 4, 0, 0, N, 60_000)
        assert d.min() >= 0 and d.max() < N
        if N <= 10:
            assert stats.chisquare(np.bincount(d, minlength=N)).pvalue > 1e-4
        else:
            # uniformity over 20 equal-probability groups
            counts = np.bincount((d.astype(np.int64) * 20) // N, minlength=20)
            expect = np.array([((g + 1) * N + 19) // 20 - (g * N + 19) // 20 for g in range(20)]) / N * len(d)
            assert stats.chisquare(counts, expect).pvalue > 1e-4


def test_bounded_rejection_heavy_range():
    # N = 2^31 + 1 rejects almost half of the words; results stay in range and unbiased.
    N = 2**31 + 1
    d = oracle.bounded_draws(7, 0, 0, 0, N, 50_000).astype(np.float64)
    assert d.max() < N
    assert abs(d.mean() / N - 0.5) < 0.01
    counts = np.bincount((d // (N / 16)).astype(np.int64), minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_bounded_unbiased_where_truncation_is_worst():
    # N = ceil(2^33 / 3): 2^32 / N = 1.5, so the multiply-shift map without its
    # rejection step gives every even value two words and every odd value one
    # (two thirds of the draws even).  With rejection every value has the same
    # number of accepted words: half even, within sampling error.
    N = 0xAAAAAAAB
    d = oracle.bounded_draws(5, 0, 0, 0, N, 40_000).astype(np.int64)
    assert d.max() < N
    assert abs(np.mean(d % 2 == 0) - 0.5) < 0.015


def test_oracle_philox_known_answers():
    """The published Philox4x32-10 known-answer vectors (tests/golden): a swapped
    output word, a key bumped before the first round or a wrong multiplier all
    fail here."""
    from kat import philox_kat
    rows = philox_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert np.array_equal(oracle.philox4x32_10(ctr, key), want), (ctr, key)


def test_input_generator_philox_known_answers():
    from kat import philox_kat
    for ctr, key, want in philox_kat():
        seed = (int(key[1]) << 32) | int(key[0])
        got = datagen._philox_blocks(np.array([ctr[0]], dtype=np.uint64), int(ctr[1]), int(ctr[2]), int(ctr[3]),
                                     seed)[0]
        assert np.array_equal(got, want), (ctr, key)


def test_stream_words_follow_the_known_answers():
    """The oracle's word stream (seed, c0, c1, c2) starts with block c3 = 0: the
    all-zero vector is the first four words of stream (0, 0, 0, 0)."""
    from kat import philox_kat
    ctr, key, want = philox_kat()[0]
    assert not ctr.any() and not key.any()
    assert np.array_equal(oracle.stream_words(0, 0, 0, 0, 4), want)
