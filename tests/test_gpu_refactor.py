"""az_refactor (a new test matrix on a resident setup) through the C ABI: its
sketch and factorisation run on the setup's own stream and overlap the next
solve's first Z* pass, so the results must not depend on that overlap.  A
refactored setup gives the same solution as a fresh setup with the same seed,
on the caller's stream and on another stream, and az_get_info / az_get_array
see the new factors."""
import numpy as np
import pytest

import workloads as W
from oracle.az import relres
from oracle.operators import Operator

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def az():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as m
    return m


def _gu():
    from tests import gpu_util
    return gpu_util


def _solve(az, gu, h, b, n, stream=None):
    x = torch.zeros((b.shape[1], n), dtype=torch.float64, device=gu.dev())
    bd = gu.to_dev_cols(b)
    if stream is not None:
        # the caller orders its own streams (inputs, index map and symbol of
        # the refactor); the factorisation itself is waited for by the library
        torch.cuda.current_stream().synchronize()
    az.az_solve(h, bd, x, stream=stream)
    if stream is not None:
        stream.synchronize()
    return gu.from_dev_cols(x)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_refactor_matches_fresh_setup(az, prec):
    gu = _gu()
    P = az.AZ_MIXED if prec == "mixed" else az.AZ_FP64
    p = W.config2(1 << 16, 8)
    op = Operator(p.grid, p.mask)
    b = p.rhs()
    fresh = {}
    for seed in (1, 2):
        h = gu.setup(p, P, seed=seed)
        try:
            fresh[seed] = (_solve(az, gu, h, b, op.N), az.az_get_info(h)["rank"])
        finally:
            az.az_destroy(h)
    h = gu.setup(p, P, seed=1)
    try:
        side = torch.cuda.Stream()
        for it, seed in enumerate((2, 1, 2, 2, 1)):
            az.az_refactor(h, seed)
            if it == 3:
                # consumers before any solve: info and arrays wait for the factors
                assert az.az_get_info(h)["rank"] == fresh[seed][1]
                sig = torch.zeros((1, fresh[seed][1]), dtype=torch.float64, device=gu.dev())
                az.az_get_array(h, az.AZ_ARRAY_SIGMA, sig)
                assert np.all(sig.cpu().numpy() > 0)
            x = _solve(az, gu, h, b, op.N, stream=side if it == 2 else None)
            assert np.array_equal(x, fresh[seed][0]), (it, seed, np.abs(x - fresh[seed][0]).max())
            assert az.az_get_info(h)["rank"] == fresh[seed][1]
    finally:
        az.az_destroy(h)
    r = relres(op, fresh[1][0], b)
    assert np.all(r < 2e-4)


def test_refactor_loop_2d(az):
    gu = _gu()
    p = W.config3(n=32, k=64)
    op = Operator(p.grid, p.mask)
    b = p.rhs()
    h0 = gu.setup(p, az.AZ_MIXED, seed=5)
    try:
        ref = _solve(az, gu, h0, b, op.N)
    finally:
        az.az_destroy(h0)
    h = gu.setup(p, az.AZ_MIXED, seed=9)
    try:
        for _ in range(3):
            az.az_refactor(h, 9)
            az.az_refactor(h, 5)          # two refactors without a solve between them
            x = _solve(az, gu, h, b, op.N)
            assert np.array_equal(x, ref)
    finally:
        az.az_destroy(h)
