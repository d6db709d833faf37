"""Pins for the oracle's Philox4x64-10 and probe rule.

The generator is checked against numpy's Philox bit generator, an independent
library implementation of the same published algorithm (Salmon et al., SC'11).
numpy's generator increments its counter before producing each 4-word block,
so a generator started at counter c - 1 yields the block for counter c.
"""
import numpy as np
import pytest

from oracle.philox import philox4x64_10, probe_bits, rademacher_probes


def _numpy_block(ctr, key):
    c = [int(x) for x in ctr]
    c[0] = (c[0] - 1) % (1 << 64)
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 7, 9, 11), (123456789, 987654321)),
    ((2**64 - 1, 3, 2**63, 1), (2**64 - 1, 2**40 + 17)),
    ((17, 3, 50, 0), (2, 0)),
])
def test_philox_matches_numpy(ctr, key):
    ref = _numpy_block(ctr, key)
    mine = philox4x64_10(np.array([ctr], dtype=np.uint64), key)[0]
    assert np.array_equal(ref, mine)


def test_philox_vectorised_matches_numpy():
    rng = np.random.default_rng(0)
    ctrs = rng.integers(1, 2**63, size=(64, 4), dtype=np.uint64)
    key = (0xDEADBEEFCAFEF00D, 0x0123456789ABCDEF)
    mine = philox4x64_10(ctrs, key)
    for i in range(ctrs.shape[0]):
        assert np.array_equal(mine[i], _numpy_block(ctrs[i], key))


def test_probe_bit_layout_against_numpy_words():
    # counter = (j >> 8, k, t, 0), key = (seed, 0); bit j & 255 -> word b>>6, bit b&63
    seed, t, k, D = 2, 3, 5, 700
    bits = probe_bits(seed, t, k, D)
    for blk in range((D + 255) // 256):
        words = _numpy_block((blk, k, t, 0), (seed, 0)) if blk > 0 else None
        if blk == 0:
            # numpy cannot start below counter 0: compute block 0 through counter
            # (0 - 1) mod 2^64 wrap, which numpy increments to 0 with carry.
            bg = np.random.Philox(counter=np.array([2**64 - 1, k - 1, t, 0], dtype=np.uint64),
                                  key=np.array([seed, 0], dtype=np.uint64))
            words = bg.random_raw(4)
        for b in range(256):
            j = blk * 256 + b
            if j >= D:
                break
            assert bits[j] == (int(words[b >> 6]) >> (b & 63)) & 1


def test_probes_are_pm1_and_balanced():
    P = rademacher_probes(seed=2, t=1, K=40, D=250_000)
    assert set(np.unique(P)) == {-1.0, 1.0}
    n = P.size                      # 1e7 draws
    mean = P.mean()
    assert abs(mean) < 5.0 / np.sqrt(n)          # 5 sigma of a fair sign
    # consecutive coordinates are not correlated
    c = np.mean(P[:, 1:] * P[:, :-1])
    assert abs(c) < 5.0 / np.sqrt(n)


def test_probes_fresh_per_iteration_and_probe():
    a = rademacher_probes(2, 1, 3, 4096)
    b = rademacher_probes(2, 2, 3, 4096)
    c = rademacher_probes(3, 1, 3, 4096)
    assert np.mean(a == b) < 0.55 and np.mean(a == c) < 0.55
    assert np.mean(a[0] == a[1]) < 0.55
    assert np.array_equal(a, rademacher_probes(2, 1, 3, 4096))   # deterministic
