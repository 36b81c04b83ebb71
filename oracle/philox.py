"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11, Sec. 2.2) and the Rademacher test matrix.

The paper (Sec. 3.2.3, paragraph "Low-rank solver") asks for r+p random
vectors without fixing their distribution.  The reading taken here: a
Rademacher (+1/-1) matrix R of size N x k whose bits come from Philox4x32-10, so
that the same R can be regenerated bit for bit on the GPU from (seed, column,
row) without storing it.

Bit layout (the one definition both sides implement independently):
  counter = (row // 128, column, 0, 0), key = (seed & 0xffffffff, seed >> 32);
  the 128 output bits are words w0..w3; row j uses bit (j % 32) of word
  ((j % 128) // 32); a set bit means +1, a clear bit -1.

Pinned by tests/test_oracle_philox.py against the published known-answer
vectors (tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def _round(c, k):
    # One Philox S-box round: two 32x32->64 multiplies, xor with the other words
    # and the round key, then a fixed word permutation (SC'11 Sec. 2.2).
    p0 = M0 * c[0]
    p1 = M1 * c[2]
    hi0, lo0 = (p0 >> 32) & MASK, p0 & MASK
    hi1, lo1 = (p1 >> 32) & MASK, p1 & MASK
    return [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]


def philox4x32_10(counter, key):
    """Pure-Python reference: 4-word counter, 2-word key -> 4 output words."""
    c = [int(v) & MASK for v in counter]
    k = [int(v) & MASK for v in key]
    for r in range(10):
        if r > 0:
            k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
        c = _round(c, k)
    return c


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit words."""
    c = [np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3)]
    k = [np.uint64(k0 & MASK), np.uint64(k1 & MASK)]
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    msk = np.uint64(MASK)
    s32 = np.uint64(32)
    for r in range(10):
        if r > 0:
            k = [np.uint64((int(k[0]) + W0) & MASK), np.uint64((int(k[1]) + W1) & MASK)]
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        c = [((p1 >> s32) & msk) ^ c[1] ^ k[0], p1 & msk,
             ((p0 >> s32) & msk) ^ c[3] ^ k[1], p0 & msk]
    return c


def rademacher(N: int, k: int, seed: int) -> np.ndarray:
    """R in {+1,-1}^{N x k} (float64), bits laid out as in the module docstring."""
    nblk = (N + 127) // 128
    out = np.empty((N, k), dtype=np.float64)
    blk = np.arange(nblk, dtype=np.uint64)
    rows = np.arange(N)
    word = (rows % 128) // 32
    bit = (rows % 32).astype(np.uint64)
    for col in range(k):
        w = philox4x32_10_np(blk, np.full(nblk, col, np.uint64), np.zeros(nblk, np.uint64),
                             np.zeros(nblk, np.uint64), seed & MASK, (seed >> 32) & MASK)
        words = np.stack(w, axis=1)                 # (nblk, 4)
        sel = words[rows // 128, word]
        b = (sel >> bit) & np.uint64(1)
        out[:, col] = np.where(b == 1, 1.0, -1.0)
    return out
