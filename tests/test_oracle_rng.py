"""Pins of the oracle's Rademacher probes (Section 2.1: entries +-1, equal odds)
against the published SplitMix64 definition (Steele, Lea, Flood, OOPSLA 2014)."""
import numpy as np


def test_splitmix64_reference_sequence(O):
    # SplitMix64 seeded with 0 returns mix64(k * 0x9e3779b97f4a7c15) for k = 1, 2, 3;
    # these three words are the generator's published reference outputs.
    g = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [O.mix64((k * g) % 2**64) for k in (1, 2, 3)]
    assert got == expect


def test_rademacher_definition(O):
    # z_i of probe p = +1 iff bit (p mod 64) of mix64((((p // 64) << 32) | i) ^ (seed * gamma)) is 0
    g = 0x9E3779B97F4A7C15
    for seed in (0, 1, 12345):
        for p in (0, 7, 63, 64, 2**20 + 3):
            z = O.rademacher(seed, p, 64)
            for i in (0, 1, 33, 63):
                h = O.mix64(((((p // 64) << 32) | i) ^ (seed * g)) % 2**64)
                assert z[i] == (1 if ((h >> (p % 64)) & 1) == 0 else -1)


def test_probes_sharing_a_hash_are_uncorrelated(O):
    # probes 64q .. 64q+63 take different bits of the same hash: still E[z_p z_q] = 0
    d = 100_000
    zs = [O.rademacher(3, p, d).astype(np.float64) for p in (128, 129, 191)]
    for a in range(3):
        for b in range(a + 1, 3):
            assert abs((zs[a] * zs[b]).mean()) < 4.0 / np.sqrt(d)


def test_rademacher_statistics(O):
    d = 200_000
    z = O.rademacher(0, 0, d).astype(np.float64)
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 4.0 / np.sqrt(d)
    # different probes are uncorrelated: E[z_p z_q] = 0 (E[z z^T] = I, Theorem 2.1)
    w = O.rademacher(0, 1, d).astype(np.float64)
    assert abs((z * w).mean()) < 4.0 / np.sqrt(d)
    # neighbouring entries uncorrelated
    assert abs((z[1:] * z[:-1]).mean()) < 4.0 / np.sqrt(d)
    # a different seed gives a different stream
    assert not np.array_equal(O.rademacher(1, 0, 64), O.rademacher(0, 0, 64))
