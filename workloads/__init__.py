"""Seeded synthetic inputs shared by the CPU oracle, the GPU tests and the bench.

This module holds none of the method's arithmetic (no kernel, symbol, FFT or
solve).  It only produces the *problem data* a user of the solver would bring:

* box / grid descriptions (sizes, oversampling, half-widths, shape parameter),
* the domain mask Omega on the oversampled grid (Sec. 2.3 Eq. set_X and
  Sec. 5.2 Eq. set_X_2d: the collocation points are the grid points in Omega),
* boundary points for the Poisson collocation problem (Sec. 6.2),
* right-hand sides: samples of the manufactured functions at the kept points.

Readings of the paper that fix these inputs:

* 1D membership uses an integer test with a 1e-9 slack so that an endpoint that
  falls on a grid point is kept (Omega is closed, Eq. set_X).
* 2D membership uses ``<=`` with no slack; the origin is inside.
* Boundary points are equispaced in the polar angle theta.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED = 230814490


@dataclass
class Grid:
    """Box [-T_d, T_d] per dimension with n[d] centers and s[d]-fold oversampling."""

    dim: int
    n: tuple
    s: tuple
    T: tuple
    epsh: float = 1.0          # eps * h (h = center spacing); eps = epsh / h

    @property
    def L(self):
        return tuple(int(a) * int(b) for a, b in zip(self.n, self.s))

    @property
    def h(self):
        return tuple(2.0 * t / n for t, n in zip(self.T, self.n))

    @property
    def hL(self):
        return tuple(2.0 * t / l for t, l in zip(self.T, self.L))

    @property
    def eps(self):
        # The shape parameter is tied to the center spacing of dimension 0; all
        # configurations here use equal spacing in both directions.
        return self.epsh / self.h[0]

    @property
    def N(self):
        return int(np.prod(self.n))

    @property
    def Ltot(self):
        return int(np.prod(self.L))


def grid_coords(grid: Grid, d: int, refine: int = 1) -> np.ndarray:
    """Coordinates -T + i*2T/(L*refine) of the (refined) oversampled grid along dim d."""
    Ld = grid.L[d] * refine
    return -grid.T[d] + np.arange(Ld) * (2.0 * grid.T[d] / Ld)


def interval_mask(grid: Grid, a: float, b: float, refine: int = 1) -> np.ndarray:
    """uint8 mask of grid points with a <= x <= b (closed interval, integer test)."""
    assert grid.dim == 1
    Ld = grid.L[0] * refine
    hL = 2.0 * grid.T[0] / Ld
    i0 = int(np.ceil((a + grid.T[0]) / hL - 1e-9))
    i1 = int(np.floor((b + grid.T[0]) / hL + 1e-9))
    m = np.zeros(Ld, dtype=np.uint8)
    m[max(i0, 0):min(i1, Ld - 1) + 1] = 1
    return m


def _mesh(grid: Grid, refine: int = 1):
    x = grid_coords(grid, 0, refine)
    y = grid_coords(grid, 1, refine)
    return np.meshgrid(x, y, indexing="ij")   # [ix][iy], iy contiguous


def disc_mask(grid: Grid, radius: float, refine: int = 1) -> np.ndarray:
    X, Y = _mesh(grid, refine)
    return (X * X + Y * Y <= radius * radius).astype(np.uint8)


def star_radius(theta, r0=0.6, a=0.15, k=5):
    return r0 + a * np.cos(k * theta)


def star_mask(grid: Grid, r0=0.6, a=0.15, k=5, refine: int = 1) -> np.ndarray:
    X, Y = _mesh(grid, refine)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    return (r <= star_radius(th, r0, a, k)).astype(np.uint8)


def star_boundary(nb=2048, r0=0.6, a=0.15, k=5) -> np.ndarray:
    th = 2.0 * np.pi * np.arange(nb) / nb
    r = star_radius(th, r0, a, k)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def star_normals(nb=2048, r0=0.6, a=0.15, k=5) -> np.ndarray:
    """Outward unit normals of the curve r(theta) = r0 + a cos(k theta) at the
    points of ``star_boundary`` (the tangent rotated by -90 degrees)."""
    th = 2.0 * np.pi * np.arange(nb) / nb
    r = star_radius(th, r0, a, k)
    dr = -a * k * np.sin(k * th)
    tx = dr * np.cos(th) - r * np.sin(th)
    ty = dr * np.sin(th) + r * np.cos(th)
    nrm = np.hypot(tx, ty)
    return np.stack([ty / nrm, -tx / nrm], axis=1)


def kept_points(grid: Grid, mask: np.ndarray, refine: int = 1) -> np.ndarray:
    """Coordinates of the kept grid points in lexicographic (x-major) order: (M, dim)."""
    if grid.dim == 1:
        return grid_coords(grid, 0, refine)[np.flatnonzero(mask)][:, None]
    X, Y = _mesh(grid, refine)
    sel = mask.reshape(-1).astype(bool)
    return np.stack([X.reshape(-1)[sel], Y.reshape(-1)[sel]], axis=1)


# ---------------------------------------------------------------------------
# The five workloads (sizes, domains, right-hand sides)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    grid: Grid
    mask: np.ndarray
    k: int
    funcs: list = field(default_factory=list)      # callables f(points)->values
    boundary: np.ndarray | None = None             # (M_b, 2) for collocation
    bfuncs: list = field(default_factory=list)     # boundary data g(points)
    weight: float = 1.0
    kind: str = "approx"                            # "approx" | "poisson"
    exact: list = field(default_factory=list)      # exact solutions (poisson)
    k0: float = 0.0                                 # Helmholtz wavenumber of the collocation operator
    normals: np.ndarray | None = None               # (M_b, dim) outward unit normals; zero row = Dirichlet
    nfuncs: list = field(default_factory=list)     # Neumann data du/dn(points, normals)

    def rhs(self) -> np.ndarray:
        pts = kept_points(self.grid, self.mask)
        return np.stack([f(pts) for f in self.funcs], axis=1)

    def boundary_rhs(self) -> np.ndarray | None:
        """Boundary data: u on Dirichlet points, du/dn on Neumann points."""
        if self.boundary is None:
            return None
        out = np.stack([g(self.boundary) for g in self.bfuncs], axis=1)
        if self.normals is not None:
            nb = np.any(self.normals != 0.0, axis=1)
            if nb.any():
                out[nb] = np.stack([h(self.boundary[nb], self.normals[nb]) for h in self.nfuncs], axis=1)
        return out


def config1() -> Problem:
    """1D approximation: N=256 on [-1,1], Omega=[-0.5,0.5], s=2, eps=1/h, k=20."""
    g = Grid(1, (256,), (2,), (1.0,), 1.0)
    m = interval_mask(g, -0.5, 0.5)
    f = lambda p: np.exp(p[:, 0]) * np.cos(8 * p[:, 0])
    return Problem("1d-n256", g, m, 20, [f])


def epsh_from_tau0(tau0: float) -> float:
    """Shape parameter of Eq. constant_shapeparam: eps = c N with
    c = pi / (2 T sqrt(2 log(1 + tau0^-2))); with h = 2T/N this is
    eps h = pi / sqrt(2 log(1 + tau0^-2))."""
    return math.pi / math.sqrt(2 * math.log(1 + tau0 ** -2))


def ode(n: int = 256, T: float = 1.5, k: int = 64, k0: float | None = None, weight: float = 10.0,
        tau0: float = 1e-10) -> Problem:
    """1D ODE of Example 6.1: u'' + k0^2 u = 0 on [-1, 1], u(+-1) = sin(+-k0), solution
    sin(k0 x) with k0 = n / 5 by default (the paper's choice), s = 2, T = 1.5 and the
    shape parameter of Eq. constant_shapeparam at tau0 = 1e-10 (Fig. d1_ode_nonper)."""
    k0 = n / 5.0 if k0 is None else float(k0)
    g = Grid(1, (n,), (2,), (T,), epsh_from_tau0(tau0))
    m = interval_mask(g, -1.0, 1.0)
    u = lambda p: np.sin(k0 * p[:, 0])
    f = lambda p: np.zeros(p.shape[0])
    return Problem(f"1d-ode-n{n}", g, m, k, [f], np.array([[-1.0], [1.0]]), [u], weight, "poisson", [u], k0)


def ode_neumann(n: int = 256, T: float = 1.5, k: int = 64, weight: float = 10.0, tau0: float = 1e-10) -> Problem:
    """Example 6.1 with a Neumann condition at the right end: u(-1) = sin(-k0),
    u'(1) = k0 cos(k0); the solution is still sin(k0 x), k0 = n / 5."""
    p = ode(n, T, k, None, weight, tau0)
    k0 = p.k0
    p.name = f"1d-ode-neumann-n{n}"
    p.normals = np.array([[0.0], [1.0]])
    p.nfuncs = [lambda q, nv: nv[:, 0] * k0 * np.cos(k0 * q[:, 0])]
    return p


def helmholtz_mixed_bc(n: int = 16, nb: int = 64, k: int = 600, k0: float = 6.0, weight: float = 10.0,
                       epsh: float = 0.5) -> Problem:
    """The Helmholtz problem on the star with Neumann data du/dn on every other
    boundary point and Dirichlet data on the rest, u = sin(pi x)cos(pi y), at
    eps h = 0.5 (where the collocation solution is accurate to ~1e-10 at n = 16;
    at eps h = 1 the saturated residual leaves O(1) errors in u)."""
    p = helmholtz(n, nb, k, k0, weight)
    p.grid = Grid(2, (n, n), (2, 2), (1.0, 1.0), epsh)
    p.name = f"2d-star-helmholtz-mixedbc-n{n}"
    nrm = star_normals(nb)
    nrm[1::2] = 0.0
    p.normals = nrm
    du = lambda q, nv: np.pi * (nv[:, 0] * np.cos(np.pi * q[:, 0]) * np.cos(np.pi * q[:, 1])
                                - nv[:, 1] * np.sin(np.pi * q[:, 0]) * np.sin(np.pi * q[:, 1]))
    p.nfuncs = [du]
    return p


def flower(n: int = 128, n_outer: int = 200, n_inner: int = 100, k: int = 1024, weight: float = 10.0,
           r0: float = 0.68, a: float = 0.2, petals: int = 5, hole: float = 0.1) -> Problem:
    """Stand-in for the flower-domain problem of Sec. 6.3: lap u + 4 u =
    exp(-4((x+0.3)^2 + y^2)^2) on a flower r <= r0 + a cos(5 theta) with a disc
    of diameter 0.2 removed, du/dn = 0 on the outer boundary (200 points),
    u = 0 on the inner one (100 points), [-1,1]^2, s = 2, eps = 1/h.  The
    paper does not give the flower's shape: r0 and a are chosen so that at
    100 x 100 centers the kept grid has about the paper's 14771 points, and the
    hole is centered at the origin.  In the operator's sign, -(lap + k0^2) u = f
    with k0 = 2 and f = -exp(...)."""
    g = Grid(2, (n, n), (2, 2), (1.0, 1.0), 1.0)
    X, Y = _mesh(g)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    m = ((r <= star_radius(th, r0, a, petals)) & (r > hole)).astype(np.uint8)
    outer = star_boundary(n_outer, r0, a, petals)
    ti = 2.0 * np.pi * np.arange(n_inner) / n_inner
    inner = np.stack([hole * np.cos(ti), hole * np.sin(ti)], axis=1)
    bpts = np.concatenate([outer, inner], axis=0)
    nrm = np.concatenate([star_normals(n_outer, r0, a, petals), np.zeros((n_inner, 2))], axis=0)
    f = lambda q: -np.exp(-4.0 * ((q[:, 0] + 0.3) ** 2 + q[:, 1] ** 2) ** 2)
    zero = lambda q: np.zeros(q.shape[0])
    p = Problem(f"2d-flower-n{n}", g, m, k, [f], bpts, [zero], weight, "poisson", [], 2.0)
    p.normals = nrm
    p.nfuncs = [lambda q, nv: np.zeros(q.shape[0])]
    return p


def helmholtz(n: int = 16, nb: int = 64, k: int = 64, k0: float = 6.0, weight: float = 10.0) -> Problem:
    """2D Helmholtz -(Lap + k0^2) u = f on the config-4 star, u = sin(pi x)cos(pi y)."""
    g = Grid(2, (n, n), (2, 2), (1.0, 1.0), 1.0)
    m = star_mask(g)
    u = lambda p: np.sin(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])
    f = lambda p: (2 * np.pi ** 2 - k0 ** 2) * np.sin(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])
    return Problem(f"2d-star-helmholtz-n{n}", g, m, k, [f], star_boundary(nb), [u], weight, "poisson", [u], k0)


def cos_family(nrhs: int, seed: int = SEED):
    rng = np.random.default_rng(seed)
    w = rng.uniform(1.0, 40.0, nrhs)
    ph = rng.uniform(0.0, 2 * np.pi, nrhs)
    return [(lambda p, a=a, b=b: np.cos(a * p[:, 0] + b)) for a, b in zip(w, ph)]


def config2(N: int = 2 ** 20, nrhs: int = 64) -> Problem:
    """1D at scale: Omega=[-0.7,0.3], s=2, eps=1/h, k=24, cos(w x + phi) RHS."""
    g = Grid(1, (N,), (2,), (1.0,), 1.0)
    m = interval_mask(g, -0.7, 0.3)
    return Problem(f"1d-n{N}", g, m, 24, cos_family(nrhs))


def config3(n: int = 256, k: int = 1024) -> Problem:
    """2D approximation on the disc |x|<=0.8 in [-1,1]^2, s=2, eps=1/h."""
    g = Grid(2, (n, n), (2, 2), (1.0, 1.0), 1.0)
    m = disc_mask(g, 0.8)
    f = lambda p: np.sin(3 * p[:, 0]) * np.exp(-p[:, 1] ** 2) + p[:, 0] * p[:, 1]
    return Problem(f"2d-disc-n{n}", g, m, k, [f])


def config4(n: int = 128, nb: int = 2048, k: int = 2048, weight: float = 10.0) -> Problem:
    """2D Poisson -Lap u = f on the star r=0.6+0.15cos(5 theta), u=sin(pi x)cos(pi y)."""
    g = Grid(2, (n, n), (2, 2), (1.0, 1.0), 1.0)
    m = star_mask(g)
    u = lambda p: np.sin(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])
    f = lambda p: 2 * np.pi ** 2 * np.sin(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])
    return Problem(f"2d-star-poisson-n{n}", g, m, k, [f], star_boundary(nb), [u],
                   weight, "poisson", [u])
