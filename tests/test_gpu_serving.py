"""Serving loop on the GPU: results alone vs in the mix, admission, a short stream."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300.serving as serving
    return serving


def _small_pool(S):
    th = 2 * np.pi * np.arange(128) / 128
    r = 0.5 + 0.1 * np.cos(5 * th)
    return [
        S.SetupSpec(("1d", 4096, -0.6), 1, (4096,), (2,), (1.0,), "approx", lambda x: (x >= -0.6) & (x <= 0.4), k=24),
        S.SetupSpec(("1d", 8192, -0.3), 1, (8192,), (2,), (1.0,), "approx", lambda x: (x >= -0.3) & (x <= 0.7), k=24),
        S.SetupSpec(("2d", 64, 0.1, 5), 2, (64, 64), (2, 2), (1.0, 1.0), "approx", S.star_fn(0.5, 0.1, 5), k=48),
        S.SetupSpec(("poisson", 64, 0.1, 5), 2, (64, 64), (2, 2), (1.0, 1.0), "poisson", S.star_fn(0.5, 0.1, 5),
                    np.stack([r * np.cos(th), r * np.sin(th)], 1), 10.0, k=48),
    ]


def _relres(az, st, x, b):
    y = torch.zeros_like(b)
    az.az_apply_A(st.h, x, y)
    return (torch.linalg.norm(y - b, dim=1) / torch.linalg.norm(b, dim=1)).cpu().numpy()


def test_each_result_is_the_same_alone_and_in_the_mix(S):
    import paper_2308_14490_gb300 as az
    pool = _small_pool(S)
    rng = np.random.default_rng(3)
    reqs = [S.Request(i, 0.0, pool[int(rng.integers(0, 4))], int(rng.integers(1, 9)), int(rng.integers(0, 2 ** 31)))
            for i in range(24)]
    mix = S.Server(8 << 30, nslots=3, keep_results=True)
    summary = mix.run(reqs, realtime=False)
    assert summary["served"] == len(reqs) and summary["rejected"] == 0
    alone = S.Server(8 << 30, nslots=1, keep_results=True)
    for r in reqs:
        single = S.Request(r.rid, 0.0, r.spec, r.nrhs, r.seed)
        alone.run([single], realtime=False)
        st = alone.setups[r.spec.key]
        rows = st.info["M"] + st.info["Mb"]
        b = torch.zeros((r.nrhs, rows), dtype=torch.float64, device=alone.dev)
        alone._rhs(st, [r], b)
        if r.spec.kind == "poisson":
            # the rows az_collocate solves: f / (2 eps^2) and w g
            eps = r.spec.epsh / (2 * r.spec.T[0] / r.spec.n[0])
            b[:, :st.info["M"]] /= 2 * eps * eps
            b[:, st.info["M"]:] *= r.spec.weight
        x_mix, x_one = mix.results[r.rid], alone.results[r.rid]
        rm, ro = _relres(az, st, x_mix, b), _relres(az, st, x_one, b)
        # the mixed-precision bar, 1e-8, for every kind of request (2D setups
        # sketch in FP64; Poisson requests go through az_collocate)
        assert np.all(np.abs(rm - ro) <= 1e-8), (r.spec.key, rm, ro)
    mix.close()
    alone.close()


def test_admission_rejects_setups_over_budget(S):
    pool = _small_pool(S)
    reqs = [S.Request(i, 0.0, pool[i % 4], 2, i) for i in range(8)]
    srv = S.Server(1 << 20, nslots=2)
    summary = srv.run(reqs, realtime=False)
    assert summary["rejected"] == 8 and summary["served"] == 0
    srv.close()


def test_short_stream_with_eviction(S):
    pool = _small_pool(S)
    reqs = S.poisson_stream(11, 100.0, 1.0, pool)
    srv = S.Server(900 << 20, nslots=4)   # room for a few setups only: forces LRU eviction
    summary = srv.run(reqs, realtime=True)
    assert summary["served"] + summary["rejected"] == len(reqs)
    assert summary["served"] > 0.9 * len(reqs)
    assert summary["latency_ms"]["p99"] is not None
    srv.close()
