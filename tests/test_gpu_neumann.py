"""Neumann boundary rows (Sec. 6.3) through the C ABI against the oracle: the
rows of A, FP64 residual parity, the error against closed-form solutions (the
ODE of Example 6.1 with a Neumann end, the star with alternating conditions),
the mixed path at eps h = 1, and the flower-with-hole stand-in."""
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


def _op(p):
    return Operator(p.grid, p.mask, "poisson", p.boundary, p.weight, k0=p.k0, normals=p.normals)


def _solve(az, gu, p, op, prec, tau, refine=-1, k=None, evaluate=0):
    h = gu.setup(p, prec, k=k, seed=11, tau=tau, refine=refine)
    try:
        xs = np.random.default_rng(3).standard_normal((op.N, 2))
        y = torch.zeros((2, op.M + op.Mb), dtype=torch.float64, device=gu.dev())
        az.az_apply_A(h, gu.to_dev_cols(xs), y)
        ref = op.A(xs)
        assert np.abs(gu.from_dev_cols(y) - ref).max() <= 1e-12 * np.abs(ref).max()
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_collocate(h, gu.to_dev_cols(p.rhs()), gu.to_dev_cols(p.boundary_rhs()), x)
        vals = None
        if evaluate:
            npts = op.N * evaluate ** p.grid.dim
            v = torch.zeros((1, npts), dtype=torch.float64, device=gu.dev())
            az.az_evaluate(h, x, evaluate, v)
            vals = gu.from_dev_cols(v)[:, 0]
        return gu.from_dev_cols(x), vals
    finally:
        az.az_destroy(h)


@pytest.mark.parametrize("n", [128, 512])
def test_ode_neumann_end(az, n):
    gu = _gu()
    p = W.ode_neumann(n=n, k=64)
    op = _op(p)
    b = op.collocation_rhs(p.rhs(), p.boundary_rhs())
    xg, vals = _solve(az, gu, p, op, az.AZ_FP64, 1e-12, refine=0, evaluate=4)
    r_o = relres(op, AZ(op, p.k, 11, 1e-12).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist())
    gf = W.Grid(1, p.grid.n, (4,), p.grid.T, p.grid.epsh)
    xf = W.grid_coords(gf, 0)
    inside = (xf >= -1.0) & (xf <= 1.0)
    assert np.abs(vals - np.sin(p.k0 * xf))[inside].max() < 1e-8


def test_star_alternating_conditions_fp64(az):
    gu = _gu()
    p = W.helmholtz_mixed_bc(n=16, nb=64)          # eps h = 0.5, k = 600 (Householder path)
    op = _op(p)
    b = op.collocation_rhs(p.rhs(), p.boundary_rhs())
    xg, _ = _solve(az, gu, p, op, az.AZ_FP64, 1e-12, refine=0)
    r_o = relres(op, AZ(op, p.k, 11, 1e-12).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist())
    ev = Operator(p.grid, p.mask)
    u = p.exact[0](W.kept_points(p.grid, p.mask))
    assert np.abs(ev.Ac(xg)[ev.idx, 0] - u).max() < 1e-8


def test_star_alternating_conditions_mixed_eps_h_1(az):
    # 2D mixed at eps h = 1: FP64 sketch (Neumann rows included), FP32 solve
    # with one FP64-residual refinement
    gu = _gu()
    p = W.helmholtz_mixed_bc(n=16, nb=64, k=64, epsh=1.0)
    op = _op(p)
    b = op.collocation_rhs(p.rhs(), p.boundary_rhs())
    x64, _ = _solve(az, gu, p, op, az.AZ_FP64, 1e-8)
    x32, _ = _solve(az, gu, p, op, az.AZ_MIXED, 1e-8)
    r_o = relres(op, AZ(op, p.k, 11, 1e-8).solve(b), b)
    r64, r32 = relres(op, x64, b), relres(op, x32, b)
    assert np.all(np.abs(r64 - r_o) <= 1e-10), (r64.tolist(), r_o.tolist())
    # the mixed solve refines once: compare with the oracle refined once
    r_o1 = relres(op, AZ(op, p.k, 11, 1e-8).solve(b, refine=1), b)
    assert np.all(np.abs(r32 - r_o1) <= 1e-8), (r32.tolist(), r_o1.tolist())


def test_flower_with_hole_parity(az):
    # Sec. 6.3 stand-in: Neumann outer boundary, Dirichlet hole, k0 = 2; the
    # sketch width equals N, so the perturbation is fully resolved
    gu = _gu()
    p = W.flower(n=32, n_outer=200, n_inner=100, k=1024)
    op = _op(p)
    b = op.collocation_rhs(p.rhs(), p.boundary_rhs())
    xg, _ = _solve(az, gu, p, op, az.AZ_FP64, 1e-10, refine=0)
    r_o = relres(op, AZ(op, p.k, 11, 1e-10).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10 + 1e-8 * r_o), (r_g.tolist(), r_o.tolist())
