"""Pins for oracle.operators against definitions written out entry by entry."""
import numpy as np
import pytest

import workloads as W
from oracle import rbf
from oracle.operators import Operator


def _phi_per(x, eps, T, deriv=0):
    f = rbf.phi if deriv == 0 else rbf.d2phi
    return sum(f(x - 2 * T * p, eps) for p in range(-30, 31))


def test_dense_Ac_1d_from_coordinates():
    # Eq. matrix_entries with explicit centers (set_centers) and grid (set_Xtilde).
    g = W.Grid(1, (12,), (3,), (1.5,), 0.7)
    op = Operator(g, np.ones(g.Ltot, np.uint8))
    A = op.Ac_dense()
    T, N, L = 1.5, 12, 36
    for i in range(L):
        for j in range(N):
            xi = -T + i * 2 * T / L
            cj = -T + j * 2 * T / N
            assert abs(A[i, j] - _phi_per(xi - cj, g.eps, T)) < 1e-15


def test_dense_Ac_2d_ordering_and_entries():
    # Sec. 5.1: j = jx*Ny + jy, basis phi_x(x - cx) phi_y(y - cy).
    g = W.Grid(2, (4, 6), (2, 2), (1.0, 1.3), 0.8)
    g.epsh = 0.8
    op = Operator(g, np.ones(g.Ltot, np.uint8))
    A = op.Ac_dense()
    Lx, Ly = g.L
    rng = np.random.default_rng(0)
    for _ in range(60):
        ix, iy = rng.integers(Lx), rng.integers(Ly)
        jx, jy = rng.integers(4), rng.integers(6)
        x = -1.0 + ix * 2.0 / Lx
        y = -1.3 + iy * 2.6 / Ly
        cx = -1.0 + jx * 2.0 / 4
        cy = -1.3 + jy * 2.6 / 6
        ref = _phi_per(x - cx, g.eps, 1.0) * _phi_per(y - cy, g.eps, 1.3)
        assert abs(A[ix * Ly + iy, jx * 6 + jy] - ref) < 1e-15


def test_dense_poisson_rows_from_definition():
    # Sec. 6.2: -(phi''(x)phi(y) + phi(x)phi''(y)) / (2 eps^2), k0 = 0.
    g = W.Grid(2, (6, 6), (2, 2), (1.0, 1.0), 1.0)
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind="poisson")
    A = op.Ac_dense()
    e = g.eps
    for (ix, iy, jx, jy) in [(0, 0, 0, 0), (3, 5, 1, 2), (11, 2, 5, 5), (7, 7, 3, 4)]:
        x = -1 + ix * 2 / 12
        y = -1 + iy * 2 / 12
        cx = -1 + jx * 2 / 6
        cy = -1 + jy * 2 / 6
        ref = -(_phi_per(x - cx, e, 1.0, 2) * _phi_per(y - cy, e, 1.0)
                + _phi_per(x - cx, e, 1.0) * _phi_per(y - cy, e, 1.0, 2)) / (2 * e * e)
        assert abs(A[ix * 12 + iy, jx * 6 + jy] - ref) < 1e-13


def test_dense_helmholtz_rows_from_definition():
    # Sec. 6.2 with k0 != 0: -(phi''(x)phi(y) + phi(x)phi''(y) + k0^2 phi(x)phi(y)) / (2 eps^2).
    g = W.Grid(2, (6, 6), (2, 2), (1.0, 1.0), 1.0)
    k0 = 7.3
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind="poisson", k0=k0)
    A = op.Ac_dense()
    e = g.eps
    for (ix, iy, jx, jy) in [(0, 0, 0, 0), (3, 5, 1, 2), (11, 2, 5, 5), (7, 7, 3, 4)]:
        x = -1 + ix * 2 / 12
        y = -1 + iy * 2 / 12
        cx = -1 + jx * 2 / 6
        cy = -1 + jy * 2 / 6
        px, py = _phi_per(x - cx, e, 1.0), _phi_per(y - cy, e, 1.0)
        ref = -(_phi_per(x - cx, e, 1.0, 2) * py + px * _phi_per(y - cy, e, 1.0, 2) + k0 ** 2 * px * py) / (2 * e * e)
        assert abs(A[ix * 12 + iy, jx * 6 + jy] - ref) < 1e-13


def test_helmholtz_fft_forms_equal_dense():
    g = W.Grid(2, (8, 8), (2, 2), (1.0, 1.0), 1.0)
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind="poisson", k0=5.0)
    a = np.random.default_rng(6).standard_normal((g.N, 3))
    d = op.Ac_dense() @ a
    assert np.abs(op.Ac(a) - d).max() <= 1e-13 * np.abs(d).max()
    opm = Operator(g, W.disc_mask(g, 0.75), kind="poisson", boundary=W.star_boundary(10), weight=3.0, k0=5.0)
    y = np.random.default_rng(7).standard_normal((opm.M + opm.Mb, 2))
    ref = opm.Zstar_dense() @ y
    assert np.abs(opm.Zstar(y) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_dense_ode_rows_from_definition():
    # Example 6.1: interior rows -(phi'' + k0^2 phi) / (2 eps^2); Dirichlet rows w phi at x = -1, 1.
    g = W.Grid(1, (24,), (2,), (1.5,), 1.0)
    k0 = 4.2
    op = Operator(g, W.interval_mask(g, -1.0, 1.0), kind="poisson", boundary=np.array([[-1.0], [1.0]]),
                  weight=10.0, k0=k0)
    Ac = op.Ac_dense()
    e = g.eps
    for (i, j) in [(0, 0), (5, 3), (47, 23), (20, 11)]:
        x = -1.5 + i * 3.0 / 48
        c = -1.5 + j * 3.0 / 24
        ref = -(_phi_per(x - c, e, 1.5, 2) + k0 ** 2 * _phi_per(x - c, e, 1.5)) / (2 * e * e)
        assert abs(Ac[i, j] - ref) < 1e-13 * max(1.0, abs(ref))
    A = op.A_dense()
    for bi, xb in enumerate((-1.0, 1.0)):
        for j in (0, 7, 23):
            c = -1.5 + j * 3.0 / 24
            assert abs(A[op.M + bi, j] - 10.0 * _phi_per(xb - c, e, 1.5)) < 1e-14
    a = np.random.default_rng(8).standard_normal((g.N, 2))
    assert np.abs(op.A(a) - A @ a).max() <= 1e-13 * np.abs(A @ a).max()
    y = np.random.default_rng(9).standard_normal((op.M + op.Mb, 2))
    ref = op.Zstar_dense() @ y
    assert np.abs(op.Zstar(y) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_boundary_rows_from_definition():
    g = W.Grid(2, (8, 8), (2, 2), (1.0, 1.0), 1.0)
    pts = W.star_boundary(16)
    op = Operator(g, W.star_mask(g), kind="poisson", boundary=pts, weight=10.0)
    A = op.A_dense()
    Ab = A[op.M:]
    for b in range(16):
        for j in [0, 9, 27, 63]:
            jx, jy = divmod(j, 8)
            cx, cy = -1 + jx * 0.25, -1 + jy * 0.25
            ref = 10.0 * _phi_per(pts[b, 0] - cx, g.eps, 1.0) * _phi_per(pts[b, 1] - cy, g.eps, 1.0)
            assert abs(Ab[b, j] - ref) < 1e-14


CASES = [
    ("1d", W.Grid(1, (32,), (2,), (1.0,), 1.0), "approx"),
    ("1d-s3", W.Grid(1, (20,), (3,), (1.5,), 0.6), "approx"),
    ("2d", W.Grid(2, (8, 12), (2, 2), (1.0, 1.0), 1.0), "approx"),
    ("2d-poisson", W.Grid(2, (8, 8), (2, 2), (1.0, 1.0), 1.0), "poisson"),
]


@pytest.mark.parametrize("name,g,kind", CASES)
def test_fft_Ac_equals_dense(name, g, kind):
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind=kind)
    a = np.random.default_rng(1).standard_normal((g.N, 3))
    d = op.Ac_dense() @ a
    assert np.abs(op.Ac(a) - d).max() <= 1e-13 * np.abs(d).max()


def _mask(g):
    if g.dim == 1:
        return W.interval_mask(g, -0.5, 0.3)
    return W.disc_mask(g, 0.75)


@pytest.mark.parametrize("name,g,kind", CASES)
def test_fft_Zstar_equals_pinv(name, g, kind):
    bnd = W.star_boundary(10) if kind == "poisson" else None
    op = Operator(g, _mask(g), kind=kind, boundary=bnd, weight=3.0)
    y = np.random.default_rng(2).standard_normal((op.M + op.Mb, 2))
    Zd = op.Zstar_dense()
    ref = Zd @ y
    assert np.abs(op.Zstar(y) - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name,g,kind", CASES)
def test_generalised_inverse_and_projection(name, g, kind):
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind=kind)
    Ac = op.Ac_dense()
    Z = op.Zstar_dense()
    assert np.abs(Ac @ Z @ Ac - Ac).max() <= 1e-11 * np.abs(Ac).max()
    # Lemma 4.4: A Z* is an orthogonal projection, so ||I - A Z*|| <= 1.
    opm = Operator(g, _mask(g), kind=kind)
    A = opm.A_dense()
    Zm = opm.Zstar_dense()
    sv = np.linalg.svd(np.eye(A.shape[0]) - A @ Zm, compute_uv=False)
    assert sv[0] <= 1 + 1e-10


@pytest.mark.parametrize("name,g,kind", CASES)
def test_whole_box_perturbation_vanishes(name, g, kind):
    op = Operator(g, np.ones(g.Ltot, np.uint8), kind=kind)
    R = np.random.default_rng(3).standard_normal((g.N, 4))
    AR = op.A(R)
    Y = AR - op.A(op.Zstar(AR))
    assert np.abs(Y).max() <= 1e-12 * np.abs(AR).max()


def test_tau_sym_zeroes_small_groups():
    g = W.Grid(1, (32,), (2,), (1.0,), 0.3)
    op0 = Operator(g, np.ones(g.Ltot, np.uint8), tau_sym=0.0)
    op1 = Operator(g, np.ones(g.Ltot, np.uint8), tau_sym=1e-3)
    small = op0.S <= 1e-6 * op0.S.max()
    assert small.any()
    assert np.all(op1.Sinv[small] == 0) and np.all(op1.Sinv[~small] > 0)


def _fd_neumann(op, pts, nrm, a, delta):
    """n . grad u_a(p) / eps by central differences of Dirichlet rows at p +- delta n."""
    plus = Operator(op.grid, op.mask, "poisson", pts + delta * nrm, op.weight, k0=op.k0)
    minus = Operator(op.grid, op.mask, "poisson", pts - delta * nrm, op.weight, k0=op.k0)
    return (plus.boundary_rows(a) - minus.boundary_rows(a)) / (2 * delta) / op.eps


@pytest.mark.parametrize("dim", [1, 2])
def test_neumann_rows_match_finite_differences(dim):
    # Sec. 6.3: a Neumann row is n . grad of the expansion at the boundary point;
    # central differences of the (independently pinned) Dirichlet rows along n.
    rng = np.random.default_rng(5)
    if dim == 1:
        g = W.Grid(1, (32,), (2,), (1.5,), 0.6)
        pts = np.array([[-1.0], [0.37], [1.0]])
        nrm = np.array([[-1.0], [0.0], [1.0]])
    else:
        g = W.Grid(2, (12, 12), (2, 2), (1.0, 1.0), 0.8)
        pts = W.star_boundary(9)
        nrm = W.star_normals(9)
        nrm[::3] = 0.0
    mask = np.ones(g.Ltot, np.uint8)
    op = Operator(g, mask, "poisson", pts, 10.0, normals=nrm)
    a = rng.standard_normal((g.N, 3))
    rows = op.boundary_rows(a)
    assert np.allclose(op.boundary_dense() @ a, rows, rtol=0, atol=1e-13 * np.abs(rows).max())
    nb = op.neumann
    fd = _fd_neumann(op, pts[nb], nrm[nb], a, 1e-5 / op.eps)
    assert np.abs(rows[nb] - fd).max() <= 1e-8 * np.abs(fd).max()
    dir_only = Operator(g, mask, "poisson", pts, 10.0)
    assert np.array_equal(rows[~nb], dir_only.boundary_rows(a)[~nb])
