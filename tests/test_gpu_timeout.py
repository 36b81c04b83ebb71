"""The bounded waits of the tensor-core projection: a wait that runs out is
reported as AZ_ERR_TIMEOUT, and the next call succeeds.

The failure is made by the library's test hook, not by a fault: the next
launch of the projection kernel stops issuing its TMA copies at a given
pipeline iteration, with every wait bounded by a few milliseconds.  The
consumers' waits then run out; each CTA stops issuing work, waits (bounded)
for its own copies and MMAs, frees its tensor memory and returns.  Nothing
traps, hangs or touches memory out of bounds.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def az():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as m
    return m


def test_tc_wait_timeout_is_reported_and_recovered(az):
    from tests import gpu_util as gu
    p = W.config2(N=1 << 16, nrhs=4)          # 1D mixed: the projection runs on the tensor cores
    g = p.grid
    mask = torch.from_numpy(p.mask).to(gu.dev())
    b = gu.to_dev_cols(p.rhs())
    opts = az.make_options(az.AZ_MIXED, 24, 1e-8, 0.0, 3, 1)
    h = az.az_setup(az.make_grid(1, g.n, g.s, g.T), mask, g.eps, options=opts)
    try:
        x = torch.zeros((4, g.N), dtype=torch.float64, device=gu.dev())
        clean = az.az_solve(h, b, x, relres=True)
        x_clean = x.clone()
        # 2048 blocks of 32 rows over up to 152 CTAs: every CTA has >= 13
        # iterations, so stopping at iteration 2 starves every CTA
        az.az_debug_tc_withhold(2, 2_000_000)
        with pytest.raises(az.AZError) as ei:
            az.az_solve(h, b, x, relres=True)
        assert ei.value.status == az.AZ_ERR_TIMEOUT
        assert "timed out" in str(ei.value)
        # the flag is reported once; the context and the handle stay usable
        again = az.az_solve(h, b, x, relres=True)
        assert np.allclose(again, clean, rtol=0, atol=1e-14)
        assert torch.equal(x, x_clean)
        info = az.az_get_info(h)
        assert info["rank"] >= 1
    finally:
        az.az_destroy(h)


def test_tc_wait_timeout_seen_by_get_info(az):
    from tests import gpu_util as gu
    p = W.config2(N=1 << 16, nrhs=2)
    g = p.grid
    mask = torch.from_numpy(p.mask).to(gu.dev())
    b = gu.to_dev_cols(p.rhs())
    opts = az.make_options(az.AZ_MIXED, 24, 1e-8, 0.0, 3, 0)
    h = az.az_setup(az.make_grid(1, g.n, g.s, g.T), mask, g.eps, options=opts)
    try:
        x = torch.zeros((2, g.N), dtype=torch.float64, device=gu.dev())
        az.az_debug_tc_withhold(0, 2_000_000)   # no copy at all
        az.az_solve(h, b, x)
        torch.cuda.synchronize()
        with pytest.raises(az.AZError) as ei:
            az.az_get_info(h)
        assert ei.value.status == az.AZ_ERR_TIMEOUT
        assert az.az_get_info(h)["rank"] >= 1
    finally:
        az.az_destroy(h)


def test_hook_rejects_bad_arguments(az):
    with pytest.raises(az.AZError) as ei:
        az.az_debug_tc_withhold(-1, 1000)
    assert ei.value.status == az.AZ_ERR_ARG
