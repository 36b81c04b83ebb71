"""Wide sketches (k > 64): Householder QR + FP64 SVD + GEMM path vs the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle.az import AZ, relres
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


def _cases():
    c1 = W.config1()
    c1.k = 100
    c3 = W.config3(n=16, k=300)          # k > N: the sketch spans everything
    c3b = W.config3(n=32, k=600)
    c4 = W.config4(n=16, nb=64, k=320)
    return [c1, c3, c3b, c4]


def _op(p):
    if p.kind == "poisson":
        return Operator(p.grid, p.mask, "poisson", p.boundary, p.weight)
    return Operator(p.grid, p.mask)


def _rhs(p, op):
    if p.kind == "poisson":
        return np.concatenate([p.rhs() / (2 * op.eps ** 2), p.weight * p.boundary_rhs()])
    return p.rhs()


@pytest.mark.parametrize("p", _cases(), ids=lambda p: f"{p.name}-k{p.k}")
def test_wide_fp64_relres_parity(az, p):
    gu = _gu()
    op = _op(p)
    b = _rhs(p, op)
    h = gu.setup(p, az.AZ_FP64, seed=13, refine=0)
    try:
        info = az.az_get_info(h)
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
        r = info["rank"]
        Ut = gu.get_array(h, az.AZ_ARRAY_UT, r, op.M + op.Mb)
        sig = torch.zeros((1, r), dtype=torch.float64, device=gu.dev())
        az.az_get_array(h, az.AZ_ARRAY_SIGMA, sig)
        sg = sig.cpu().numpy()[0]
    finally:
        az.az_destroy(h)
    ref = AZ(op, p.k, 13, 1e-8)
    assert r == ref.rank
    assert np.allclose(sg, ref.sig[:r], rtol=1e-8, atol=1e-12 * ref.sig[0])
    assert np.abs(Ut.T @ Ut - np.eye(r)).max() <= 1e-10
    r_o = relres(op, ref.solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist())


def _mixed_vs_fp64(az, p, b, refine=-1):
    gu = _gu()
    op = _op(p)
    out = {}
    for prec in (az.AZ_FP64, az.AZ_MIXED):
        h = gu.setup(p, prec, seed=13, refine=refine if prec == az.AZ_MIXED else 0)
        try:
            x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
            az.az_solve(h, gu.to_dev_cols(b), x)
            out[prec] = relres(op, gu.from_dev_cols(x), b)
        finally:
            az.az_destroy(h)
    return out[az.AZ_FP64], out[az.AZ_MIXED]


@pytest.mark.parametrize("p", _cases()[1:3], ids=lambda p: f"{p.name}-k{p.k}")
def test_wide_mixed_consistent_rhs(az, p):
    """b = A c (c seeded normal), so only the truncation leaves a residual
    (~2e-9 in FP64).  In 2D hundreds of singular values of Y lie between the
    FP32 sketch's noise floor and tau; the refined mixed solve settles a few
    1e-8 above the FP64 residual (2 steps: 3e-8 at most on these inputs, a
    third step no longer lowers it)."""
    op = _op(p)
    c = np.random.default_rng(5).standard_normal((op.N, 4))
    b = op.A(c)
    r64, r32 = _mixed_vs_fp64(az, p, b, refine=2)
    print("consistent", p.name, r64.tolist(), r32.tolist())
    assert np.all(r64 <= 1e-8)
    assert np.all(np.abs(r32 - r64) <= 5e-8), (r32.tolist(), r64.tolist())


def test_wide_mixed_unresolved_rhs(az):
    """Problem right-hand side on a coarse grid (optimal residual ~1e-4): the
    FP32 sketch's noise tilts the fitted subspace, so the mixed residual may
    exceed the optimum by a few per cent, never by orders of magnitude."""
    p = _cases()[2]
    op = _op(p)
    r64, r32 = _mixed_vs_fp64(az, p, _rhs(p, op))
    print("unresolved", r64.tolist(), r32.tolist())
    assert np.all(r32 <= 1.1 * r64)
