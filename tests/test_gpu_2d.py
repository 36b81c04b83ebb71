"""GPU parity of the 2D approximation and 2D Poisson collocation paths."""
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
    c3 = W.config3(n=16, k=48)
    c3b = W.config3(n=32, k=64)
    c3r = W.Problem("2d-rect", W.Grid(2, (16, 32), (2, 2), (1.0, 1.3), 1.0), None, 40,
                    [lambda p: np.cos(2 * p[:, 0]) * p[:, 1]])
    c3r.mask = W.star_mask(c3r.grid, 0.7, 0.2, 3)
    c4 = W.config4(n=16, nb=64, k=64)
    return [c3, c3b, c3r, c4]


def _op(p):
    if p.kind == "poisson":
        return Operator(p.grid, p.mask, "poisson", p.boundary, p.weight)
    return Operator(p.grid, p.mask)


def _rhs(p, op):
    if p.kind == "poisson":
        return np.concatenate([p.rhs() / (2 * op.eps ** 2), p.weight * p.boundary_rhs()])
    return p.rhs()


@pytest.mark.parametrize("p", _cases(), ids=lambda p: p.name)
def test_operators_fp64(az, p):
    gu = _gu()
    op = _op(p)
    h = gu.setup(p, az.AZ_FP64)
    try:
        G = gu.get_array(h, az.AZ_ARRAY_SYMBOL, 1, op.Ltot)[:, 0]
        assert np.abs(G - op.Ghat.reshape(-1)).max() <= 1e-12 * np.abs(op.Ghat).max()
        rng = np.random.default_rng(5)
        xs = rng.standard_normal((op.N, 3))
        y = torch.zeros((3, op.M + op.Mb), dtype=torch.float64, device=gu.dev())
        az.az_apply_A(h, gu.to_dev_cols(xs), y)
        ref = op.A(xs)
        assert np.abs(gu.from_dev_cols(y) - ref).max() <= 1e-12 * np.abs(ref).max()
        ys = rng.standard_normal((op.M + op.Mb, 3))
        z = torch.zeros((3, op.N), dtype=torch.float64, device=gu.dev())
        az.az_apply_Zstar(h, gu.to_dev_cols(ys), z)
        ref = op.Zstar(ys)
        assert np.abs(gu.from_dev_cols(z) - ref).max() <= 1e-11 * np.abs(ref).max()
    finally:
        az.az_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("p", _cases(), ids=lambda p: p.name)
def test_sketch_2d(az, p, prec):
    gu = _gu()
    op = _op(p)
    h = gu.setup(p, az.AZ_FP64 if prec == "fp64" else az.AZ_MIXED, seed=11)
    try:
        ref = AZ(op, p.k, 11, 1e-8)
        Wg = gu.get_array(h, az.AZ_ARRAY_W, p.k, op.N)
        Wref = ref.R - op.Zstar(op.A(ref.R))
        # (2D mixed setups sketch in FP64 as well)
        tol = 1e-11
        assert np.abs(Wg - Wref).max() <= tol * np.abs(Wref).max()
        Yg = gu.get_array(h, az.AZ_ARRAY_SKETCH, p.k, op.M + op.Mb)
        assert np.abs(Yg - ref.Y).max() <= tol * np.abs(ref.Y).max()
    finally:
        az.az_destroy(h)


@pytest.mark.parametrize("p", _cases(), ids=lambda p: p.name)
def test_solve_2d_fp64_parity(az, p):
    gu = _gu()
    op = _op(p)
    b = _rhs(p, op)
    h = gu.setup(p, az.AZ_FP64, seed=11, refine=0)
    try:
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        if p.kind == "poisson":
            f = gu.to_dev_cols(p.rhs())
            gb = gu.to_dev_cols(p.boundary_rhs())
            rr = az.az_collocate(h, f, gb, x, relres=True)
        else:
            rr = az.az_solve(h, gu.to_dev_cols(b), x, relres=True)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    r_o = relres(op, AZ(op, p.k, 11, 1e-8).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist())
    assert np.allclose(rr, r_g, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("p", _cases(), ids=lambda p: p.name)
def test_solve_2d_mixed_parity(az, p):
    """The mixed path (FP64 sketch and factors in 2D, FP32 transforms, stencils
    and projection in the solve, one FP64-residual refinement) against the
    oracle's Algorithm 1 with the same R, k, tau and one refinement: 1e-8.
    Collocation setups go through az_collocate (its row scaling)."""
    gu = _gu()
    op = _op(p)
    b = _rhs(p, op)
    h = gu.setup(p, az.AZ_MIXED, seed=11, refine=1)
    try:
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        if p.kind == "poisson":
            rr = az.az_collocate(h, gu.to_dev_cols(p.rhs()), gu.to_dev_cols(p.boundary_rhs()), x, relres=True)
        else:
            rr = az.az_solve(h, gu.to_dev_cols(b), x, relres=True)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    r_o = relres(op, AZ(op, p.k, 11, 1e-8).solve(b, refine=1), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-8), (r_g.tolist(), r_o.tolist())
    assert np.allclose(rr, r_g, rtol=1e-8, atol=1e-14)


def test_poisson_fine_grid_error(az):
    # error of u on the s_test = 4 refinement inside the star vs the oracle's
    gu = _gu()
    p = W.config4(n=16, nb=64, k=64)
    op = _op(p)
    b = _rhs(p, op)
    h = gu.setup(p, az.AZ_FP64, seed=11, refine=0)
    try:
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_collocate(h, gu.to_dev_cols(p.rhs()), gu.to_dev_cols(p.boundary_rhs()), x)
        out = torch.zeros((1, op.N * 16), dtype=torch.float64, device=gu.dev())
        az.az_evaluate(h, x, 4, out)
        vals = gu.from_dev_cols(out)[:, 0]
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    gf = W.Grid(2, p.grid.n, (4, 4), p.grid.T, p.grid.epsh)
    opf = Operator(gf, np.ones(gf.Ltot, np.uint8))
    assert np.abs(vals - opf.Ac(xg)[:, 0]).max() <= 1e-11 * max(1.0, np.abs(xg).max())
    inside = W.star_mask(gf).reshape(-1).astype(bool)
    X, Y = np.meshgrid(W.grid_coords(gf, 0), W.grid_coords(gf, 1), indexing="ij")
    u = p.exact[0](np.stack([X.reshape(-1), Y.reshape(-1)], 1))
    err_g = np.abs(vals - u)[inside].max()
    err_o = np.abs(opf.Ac(AZ(op, p.k, 11, 1e-8).solve(b))[:, 0] - u)[inside].max()
    assert err_g <= max(1.01 * err_o, err_o + 1e-9)


def test_whole_box_2d_rank_zero(az):
    gu = _gu()
    g = W.Grid(2, (16, 16), (2, 2), (1.0, 1.0), 1.0)
    p = W.Problem("box2d", g, np.ones(g.Ltot, np.uint8), 8, [lambda q: np.sin(q[:, 0] + 2 * q[:, 1])])
    op = Operator(g, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_FP64, refine=0)
    try:
        assert az.az_get_info(h)["rank"] == 0
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    z = op.Zstar(b)
    assert np.abs(xg - z).max() <= 1e-11 * np.abs(z).max()
