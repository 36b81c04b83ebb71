"""Pins for oracle.philox: published known-answer vectors and the bit layout."""
import os

import numpy as np

from oracle.philox import philox4x32_10, philox4x32_10_np, rademacher

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if line:
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        assert philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_vectorised_matches_scalar():
    rows = _kat()
    for r in rows:
        out = philox4x32_10_np(*[np.array([v], np.uint64) for v in r[0:4]], r[4], r[5])
        assert [int(o[0]) for o in out] == r[6:10]


def test_rademacher_bit_layout_bruteforce():
    seed = 0x123456789ABCDEF
    N, k = 300, 3
    R = rademacher(N, k, seed)
    for col in range(k):
        for j in range(0, N, 7):
            w = philox4x32_10([j // 128, col, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
            bit = (w[(j % 128) // 32] >> (j % 32)) & 1
            assert R[j, col] == (1.0 if bit else -1.0)


def test_rademacher_statistics():
    R = rademacher(4096, 8, 42)
    assert set(np.unique(R)) == {-1.0, 1.0}
    assert abs(R.mean()) < 0.02
    G = R.T @ R / 4096.0
    assert np.abs(G - np.eye(8)).max() < 0.06
