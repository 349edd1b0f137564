"""Reference of the library's on-device white-noise generator (Sec. 3.1, step A.1).

Test infrastructure (see ``oracle/__init__``).  The paper draws the initial white noise
from a seeded random stream; the library offers, besides taking w as an input, a device
generator built from two published definitions, restated here independently of the CUDA
code:

* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC11 2011): a 128-bit counter and a 64-bit
  key; ten rounds, each multiplying counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57
  (64-bit products split into high and low halves) and mixing the high halves with the
  other two words and the key; the key is bumped by the Weyl constants 0x9E3779B9 and
  0xBB67AE85 before every round after the first.
* Box-Muller (1958): two uniforms u0, u1 in (0, 1) give the standard normals
  sqrt(-2 ln u0) cos(2 pi u1) and sqrt(-2 ln u0) sin(2 pi u1).

Cell i of the N^3 grid (flat index, k fastest) takes word i % 4 of the block with counter
(g mod 2^32, g div 2^32, 0, 0), g = i div 4, and key (seed mod 2^32, seed div 2^32); a
word x becomes the uniform (floor(x / 2^8) + 1/2) 2^-24 (its top 24 bits: exact in FP32,
never 0 or 1); words 0, 1 and 2, 3 form the Box-Muller pairs (cos for the even word, sin
for the odd one).

Pins (tests/test_oracle_rng.py): the published known-answer vectors
(tests/golden/philox4x32_10_kat.txt); moments and independence of the normals.
"""
import numpy as np

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32-10 of one counter block (4 words) under a key (2 words) -> 4 words."""
    c0, c1, c2, c3 = (int(v) & _MASK for v in counter)
    k0, k1 = (int(v) & _MASK for v in key)
    for r in range(10):
        if r:
            k0, k1 = (k0 + _W0) & _MASK, (k1 + _W1) & _MASK
        p0, p1 = _M0 * c0, _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & _MASK, (p0 >> 32) ^ c3 ^ k1, p0 & _MASK)
    return [c0, c1, c2, c3]


def philox4x32_10_blocks(nblocks, seed):
    """Words of the blocks g = 0 .. nblocks-1 (vectorised, uint64 arithmetic), shape (nblocks, 4)."""
    g = np.arange(nblocks, dtype=np.uint64)
    c = [g & np.uint64(_MASK), g >> np.uint64(32), np.zeros_like(g), np.zeros_like(g)]
    k0, k1 = np.uint64(seed & _MASK), np.uint64((seed >> 32) & _MASK)
    m = np.uint64(_MASK)
    for r in range(10):
        if r:
            k0, k1 = (k0 + np.uint64(_W0)) & m, (k1 + np.uint64(_W1)) & m
        p0 = np.uint64(_M0) * c[0]
        p1 = np.uint64(_M1) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & m, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & m]
    return np.stack(c, axis=1)


def white_noise(N, seed):
    """The device generator's N^3 standard normals, in FP64 (flat index order, shape N^3)."""
    n = N**3
    words = philox4x32_10_blocks((n + 3) // 4, seed)
    u = ((words >> np.uint64(8)).astype(np.float64) + 0.5) / 16777216.0
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r01 * np.sin(2 * np.pi * u[:, 1]),
                  r23 * np.cos(2 * np.pi * u[:, 3]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1)
    return z.reshape(-1)[:n]
