"""The periodic problem (Omega = the whole box) through the C ABI: the
perturbation is exactly zero (Sec. 3.1), the setup skips the sketch, and the
solve is the plain inverse Z*.  The paper's periodic example (Sec. 3.3,
Fig. d1_fa_per): f = sin([N/5] pi x), T = 1, tau0 = 1e-10, maximum error below
1e-12 and ||a|| / sqrt(N) about 5 (s = 2 and 4 here; the paper uses s = 3)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.az import relres
from oracle.operators import Operator
from tests.paper_values import paper_value

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


@pytest.mark.parametrize("N,s", [(256, 2), (4096, 2), (65536, 2), (4096, 4)])
def test_paper_periodic_example(az, N, s):
    gu = _gu()
    g = W.Grid(1, (N,), (s,), (1.0,), W.epsh_from_tau0(1e-10))
    fq = math.floor(N / 5)
    f = lambda q: np.sin(fq * math.pi * q[:, 0])
    p = W.Problem(f"periodic-n{N}", g, np.ones(g.Ltot, np.uint8), 64, [f])
    op = Operator(g, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_FP64, seed=3, refine=0)
    try:
        assert az.az_get_info(h)["rank"] == 0
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
        st = 16 if N <= 4096 else 4
        vals = torch.zeros((1, op.N * st), dtype=torch.float64, device=gu.dev())
        az.az_evaluate(h, x, st, vals)
        vals = gu.from_dev_cols(vals)[:, 0]
    finally:
        az.az_destroy(h)
    z = op.Zstar(b)                     # the oracle's plain inverse
    # Z* divides each alias group by its S_k, so rounding in the transform of
    # b is amplified by up to sqrt(max S / min S) (about 1e10 at this eps h)
    amp = math.sqrt(op.S.max() / op.S.min())
    assert np.abs(xg - z).max() <= max(1e-10, 100 * 2.2e-16 * amp) * np.abs(z).max()
    gf = W.Grid(1, (N,), (st,), (1.0,), g.epsh)
    u = np.sin(fq * math.pi * W.grid_coords(gf, 0))
    err = np.abs(vals - u).max()
    if N <= 4096:
        assert err < paper_value("E1_max_error_bound")
    else:
        # rounding grows slowly with N (the oracle reaches ~5e-12 at N = 65536)
        opf = Operator(gf, np.ones(gf.Ltot, np.uint8))
        err_o = np.abs(opf.Ac(z)[:, 0] - u).max()
        assert err <= 2 * err_o + 1e-13, (err, err_o)
    assert abs(np.linalg.norm(xg) / math.sqrt(N) - paper_value("E1_coef_norm_over_sqrtN")) < 1.0


def test_whole_box_mixed_and_2d(az):
    # mixed precision at eps h = 1 (the FP32 sketch is skipped, the refined
    # solve stays within the parity bar), and a 2D whole box
    gu = _gu()
    g = W.Grid(1, (1 << 14,), (2,), (1.0,), 1.0)
    p = W.Problem("box1d", g, np.ones(g.Ltot, np.uint8), 24, W.cos_family(4))
    op = Operator(g, p.mask)
    b = p.rhs()
    out = {}
    for prec in (az.AZ_FP64, az.AZ_MIXED):
        h = gu.setup(p, prec, seed=3)
        try:
            assert az.az_get_info(h)["rank"] == 0
            x = torch.zeros((4, op.N), dtype=torch.float64, device=gu.dev())
            az.az_solve(h, gu.to_dev_cols(b), x)
            out[prec] = relres(op, gu.from_dev_cols(x), b)
        finally:
            az.az_destroy(h)
    assert np.all(np.abs(out[az.AZ_MIXED] - out[az.AZ_FP64]) <= 1e-8)
    g2 = W.Grid(2, (64, 64), (2, 2), (1.0, 1.0), 1.0)
    p2 = W.Problem("box2d", g2, np.ones(g2.Ltot, np.uint8), 64,
                   [lambda q: np.sin(3 * q[:, 0]) * np.cos(2 * q[:, 1])])
    op2 = Operator(g2, p2.mask)
    b2 = p2.rhs()
    h = gu.setup(p2, az.AZ_FP64, seed=3, refine=0)
    try:
        assert az.az_get_info(h)["rank"] == 0
        x = torch.zeros((1, op2.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b2), x)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    z = op2.Zstar(b2)
    assert np.abs(xg - z).max() <= 1e-12 * np.abs(z).max()
