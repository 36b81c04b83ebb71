"""GPU parity of the 1D hot path against the oracle (through the C ABI)."""
import numpy as np
import pytest

import workloads as W
from oracle import philox
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


def test_rademacher_bit_exact(az):
    gu = _gu()
    for (N, k, seed) in [(1, 1, 0), (300, 3, 0x123456789ABCDEF), (4096, 24, 7), (1000003 // 7, 5, 2 ** 63 + 11)]:
        R = torch.zeros((k, N), dtype=torch.float64, device=gu.dev())
        az.az_rademacher(N, k, seed, R)
        ref = philox.rademacher(N, k, seed)
        assert np.array_equal(gu.from_dev_cols(R), ref)


CASES_1D = [
    W.config1(),
    W.Problem("1d-ragged", W.Grid(1, (64,), (2,), (1.0,), 1.0), None, 9),
    W.Problem("1d-s4", W.Grid(1, (128,), (4,), (1.5,), 0.8), None, 15),
]
CASES_1D[1].mask = W.interval_mask(CASES_1D[1].grid, -0.61, 0.37)
CASES_1D[2].mask = W.interval_mask(CASES_1D[2].grid, -1.0, 1.0)
for _c in CASES_1D[1:]:
    _c.funcs = [lambda p: np.cos(5 * p[:, 0]) + p[:, 0] ** 2, lambda p: np.exp(-p[:, 0])]


@pytest.mark.parametrize("p", CASES_1D, ids=lambda p: p.name)
def test_symbol_and_operators_fp64(az, p):
    gu = _gu()
    op = Operator(p.grid, p.mask)
    h = gu.setup(p, az.AZ_FP64)
    try:
        G = gu.get_array(h, az.AZ_ARRAY_SYMBOL, 1, op.Ltot)[:, 0]
        assert np.abs(G - op.Ghat).max() <= 1e-13 * np.abs(op.Ghat).max()
        rng = np.random.default_rng(3)
        xs = rng.standard_normal((op.N, 3))
        y = torch.zeros((3, op.M), dtype=torch.float64, device=gu.dev())
        az.az_apply_A(h, gu.to_dev_cols(xs), y)
        ref = op.A(xs)
        assert np.abs(gu.from_dev_cols(y) - ref).max() <= 1e-13 * np.abs(ref).max()
        ys = rng.standard_normal((op.M, 3))
        z = torch.zeros((3, op.N), dtype=torch.float64, device=gu.dev())
        az.az_apply_Zstar(h, gu.to_dev_cols(ys), z)
        ref = op.Zstar(ys)
        assert np.abs(gu.from_dev_cols(z) - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        az.az_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("p", CASES_1D, ids=lambda p: p.name)
def test_sketch_matches_oracle(az, p, prec):
    gu = _gu()
    op = Operator(p.grid, p.mask)
    h = gu.setup(p, az.AZ_FP64 if prec == "fp64" else az.AZ_MIXED, seed=7)
    try:
        ref = AZ(op, p.k, 7, 1e-8)
        R = gu.get_array(h, az.AZ_ARRAY_R, p.k, op.N)
        assert np.array_equal(R, ref.R)
        Wg = gu.get_array(h, az.AZ_ARRAY_W, p.k, op.N)
        Wref = ref.R - op.Zstar(op.A(ref.R))
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.abs(Wg - Wref).max() <= tol * np.abs(Wref).max()
        Yg = gu.get_array(h, az.AZ_ARRAY_SKETCH, p.k, op.M)
        assert np.abs(Yg - ref.Y).max() <= tol * np.abs(ref.Y).max()
        info = az.az_get_info(h)
        r = info["rank"]
        Ut = gu.get_array(h, az.AZ_ARRAY_UT, r, op.M)
        assert np.abs(Ut.T @ Ut - np.eye(r)).max() <= (1e-10 if prec == "fp64" else 1e-5)
        sig = torch.zeros((1, r), dtype=torch.float64, device=gu.dev())
        az.az_get_array(h, az.AZ_ARRAY_SIGMA, sig)
        sg = sig.cpu().numpy()[0]
        strong = ref.sig > 1e-5 * ref.sig[0]
        n = int(strong.sum())
        # FP64: relative agreement; mixed: the FP32 sketch carries absolute noise
        # of order u_32 * sigma_1 on every singular value.
        if prec == "fp64":
            assert np.allclose(sg[:n], ref.sig[:n], rtol=1e-9)
        else:
            assert np.abs(sg[:n] - ref.sig[:n]).max() <= 1e-6 * ref.sig[0]
    finally:
        az.az_destroy(h)


@pytest.mark.parametrize("p", CASES_1D, ids=lambda p: p.name)
def test_solve_fp64_relres_parity(az, p):
    gu = _gu()
    op = Operator(p.grid, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_FP64, seed=7, refine=0)
    try:
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        rr = az.az_solve(h, gu.to_dev_cols(b), x, relres=True)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    ref = AZ(op, p.k, 7, 1e-8)
    r_o = relres(op, ref.solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist(), (r_g - r_o).tolist())
    assert np.allclose(rr, r_g, rtol=1e-9, atol=1e-15)


def test_solve_mixed_relres_parity_large(az):
    # Mixed precision (FP32 sketch/transforms) + 1 FP64-residual refinement:
    # parity bar 1e-8 holds once M is large (the FP32 noise floor of the sketch
    # enters the residual as ~1/M).
    gu = _gu()
    g = W.Grid(1, (1 << 16,), (2,), (1.0,), 1.0)
    p = W.Problem("1d-n65536", g, W.interval_mask(g, -0.5, 0.5), 24, W.cos_family(6))
    op = Operator(g, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_MIXED, seed=7)
    try:
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    r_o = relres(op, AZ(op, 24, 7, 1e-8).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-8), (r_g - r_o)


def test_whole_box_rank_zero(az):
    gu = _gu()
    g = W.Grid(1, (256,), (2,), (1.0,), 1.0)
    p = W.Problem("box", g, np.ones(g.Ltot, np.uint8), 8, [lambda q: np.sin(3 * q[:, 0])])
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
    assert np.abs(xg - z).max() <= 1e-12 * np.abs(z).max()


def test_fine_grid_error(az):
    # Max error on the s_test = 16 refinement inside Omega vs the oracle's own error.
    gu = _gu()
    p = W.config1()
    op = Operator(p.grid, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_FP64, refine=0)
    try:
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        out = torch.zeros((1, op.N * 16), dtype=torch.float64, device=gu.dev())
        az.az_evaluate(h, x, 16, out)
        vals = gu.from_dev_cols(out)[:, 0]
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    gf = W.Grid(1, p.grid.n, (16,), p.grid.T, p.grid.epsh)
    opf = Operator(gf, np.ones(gf.Ltot, np.uint8))
    assert np.abs(vals - opf.Ac(xg)[:, 0]).max() <= 1e-12 * np.abs(xg).max()
    mf = W.interval_mask(gf, -0.5, 0.5).astype(bool)
    xf = W.grid_coords(gf, 0)
    f = p.funcs[0](xf[:, None])
    err_g = np.abs(vals - f)[mf].max()
    err_o = np.abs(opf.Ac(AZ(op, p.k, 7, 1e-8).solve(b))[:, 0] - f)[mf].max()
    assert err_g <= max(1.01 * err_o, err_o + 1e-9 * np.abs(f).max())


def test_config2_scale_zstar_and_solve(az):
    """Config-2 geometry (N = 2^20, L = 2^21, s = 2, Omega = [-0.7, 0.3], k = 24,
    mixed): the same FFT-pass kernels and launch shapes the benchmark step times.
    Z* in FP32 against the oracle's FP64 FFT form, and the refined solve's relres
    against the oracle AZ with the same R, k and tau."""
    gu = _gu()
    p = W.config2(1 << 20, 4)
    op = Operator(p.grid, p.mask)
    b = p.rhs()
    h = gu.setup(p, az.AZ_MIXED, seed=1)
    try:
        ys = np.random.default_rng(11).standard_normal((op.M, 3))
        z = torch.zeros((3, op.N), dtype=torch.float64, device=gu.dev())
        az.az_apply_Zstar(h, gu.to_dev_cols(ys), z)
        ref = op.Zstar(ys)
        # FP32 transforms of length 2^21: a few hundred units of FP32 rounding
        assert np.abs(gu.from_dev_cols(z) - ref).max() <= 2e-5 * np.abs(ref).max()
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    r_o = relres(op, AZ(op, 24, 1, 1e-8).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-8), (r_g - r_o)
