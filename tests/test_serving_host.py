"""Host-side pieces of the serving loop (no GPU): the seeded workload."""
import collections

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_pool_and_stream_are_seeded_and_mixed():
    import paper_2308_14490_gb300.serving as S
    p1 = S.setup_pool(230814490)
    p2 = S.setup_pool(230814490)
    assert [s.key for s in p1] == [s.key for s in p2]
    kinds = collections.Counter(s.kind + str(s.dim) for s in p1)
    assert set(kinds) == {"approx1", "approx2", "poisson2"}
    reqs = S.poisson_stream(230814490, 200.0, 20.0, p1)
    assert abs(len(reqs) - 4000) < 4 * np.sqrt(4000)          # Poisson count at 200/s over 20 s
    gaps = np.diff([r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    assert min(r.nrhs for r in reqs) == 1 and max(r.nrhs for r in reqs) == 32
    for r in reqs[:50]:
        assert r.spec.dim in (1, 2)


def test_star_domain_mask():
    import paper_2308_14490_gb300.serving as S
    f = S.star_fn(0.5, 0.1, 5)
    X, Y = np.meshgrid(np.linspace(-1, 1, 41), np.linspace(-1, 1, 41), indexing="ij")
    m = f(X, Y)
    assert m[20, 20] and not m[0, 0]
    assert m.sum() > 0.1 * m.size and m.sum() < 0.5 * m.size
