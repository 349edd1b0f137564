"""Pins of the reference white-noise generator (Philox4x32-10 + Box-Muller)."""
import os

import numpy as np

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        yield v[0:4], v[4:6], v[6:10]


def test_published_known_answer_vectors():
    n = 0
    for ctr, key, want in _kat():
        assert rng.philox4x32_10(ctr, key) == want
        n += 1
    assert n == 3


def test_vectorised_blocks_equal_the_scalar_definition():
    seed = 0x1234_5678_9ABC_DEF0
    blocks = rng.philox4x32_10_blocks(70, seed)
    for g in (0, 1, 31, 69):
        want = rng.philox4x32_10([g & 0xFFFFFFFF, g >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert [int(v) for v in blocks[g]] == want


def test_normals_have_unit_moments_and_no_correlation():
    z = rng.white_noise(64, 7)
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(z**4) - 3.0) < 0.05
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5.0 / np.sqrt(n)
    z2 = rng.white_noise(64, 8)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5.0 / np.sqrt(n)
    # a grid that is not a multiple of 4 cells takes the first words of its last block
    assert np.array_equal(rng.white_noise(5, 3), rng.white_noise(6, 3)[:125])
