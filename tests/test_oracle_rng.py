"""Pins of the oracle's Philox4x32-10 and its uniform conversions.

Philox (Salmon et al., SC'11) is pinned two ways that do not use the
oracle's own code: the known-answer vectors published with the Random123
distribution, and a width-generic restatement of the round function that
reproduces numpy's independent Philox4x64-10 at 64 bits and the oracle at
32 bits.
"""
import numpy as np
import pytest

import oracle

M32 = (0xD2511F53, 0xCD9E8D57)
K32 = (0x9E3779B9, 0xBB67AE85)
M64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
K64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox_generic(ctr, key, W, M, K, rounds=10):
    mask = (1 << W) - 1
    c, k = list(ctr), list(key)
    for _ in range(rounds):
        p0, p1 = M[0] * c[0], M[1] * c[2]
        c = [(p1 >> W) ^ c[1] ^ k[0], p1 & mask, (p0 >> W) ^ c[3] ^ k[1], p0 & mask]
        k = [(k[0] + K[0]) & mask, (k[1] + K[1]) & mask]
    return c


KAT = [  # Random123 kat_vectors, philox4x32 10 rounds
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    assert tuple(oracle.philox4x32_10(ctr, key)) == want


def test_generic_round_function_matches_numpy_philox4x64():
    rng = np.random.default_rng(5)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 2**63, 4)]
        key = [int(x) for x in rng.integers(0, 2**63, 2)]
        bg = np.random.Philox(counter=ctr, key=key)
        raw = [int(x) for x in bg.random_raw(4)]
        # numpy advances the counter before its first block
        c1 = list(ctr)
        c1[0] = (c1[0] + 1) & ((1 << 64) - 1)
        assert raw == philox_generic(c1, key, 64, M64, K64)


def test_oracle_philox_matches_generic_at_32_bits():
    rng = np.random.default_rng(6)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2**32, 4)]
        key = [int(x) for x in rng.integers(0, 2**32, 2)]
        assert oracle.philox4x32_10(ctr, key) == philox_generic(ctr, key, 32, M32, K32)


def test_philox_outputs_are_uniform_bits():
    # bit balance over many counters (a dropped xor or a wrong multiplier skews it)
    words = np.array([oracle.philox4x32_10((i, 0, 7, 3), (11, 13)) for i in range(4000)],
                     dtype=np.uint64).ravel()
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / np.sqrt(len(words)))
