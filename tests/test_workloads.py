"""The seeded input recipes: geometry helpers and the sizes the recipes claim."""
import numpy as np

import workloads as W


def test_star_normals_are_outward_unit_normals():
    n = 97
    P = W.star_boundary(n)
    Nv = W.star_normals(n)
    assert np.allclose(np.hypot(Nv[:, 0], Nv[:, 1]), 1.0, atol=1e-14)
    # orthogonal to the curve's chord at each point (central difference of the parametrisation)
    th = 2 * np.pi * np.arange(n) / n
    d = 1e-6
    r = lambda t: W.star_radius(t)
    tang = np.stack([r(th + d) * np.cos(th + d) - r(th - d) * np.cos(th - d),
                     r(th + d) * np.sin(th + d) - r(th - d) * np.sin(th - d)], axis=1)
    assert np.abs(np.sum(tang * Nv, axis=1)).max() < 1e-8
    # outward: moving along the normal leaves the star
    out = P + 1e-3 * Nv
    rr = np.hypot(out[:, 0], out[:, 1])
    assert np.all(rr > W.star_radius(np.arctan2(out[:, 1], out[:, 0])))


def test_config2_sizes_and_flower_count():
    p = W.config2(1 << 20, 2)
    assert p.grid.Ltot == 1 << 21 and int(p.mask.sum()) == 1 << 20
    # the flower stand-in keeps about the paper's 14771 collocation points at 100 x 100 centers
    g = W.Grid(2, (100, 100), (2, 2), (1.0, 1.0), 1.0)
    X, Y = np.meshgrid(W.grid_coords(g, 0), W.grid_coords(g, 1), indexing="ij")
    r, th = np.hypot(X, Y), np.arctan2(Y, X)
    m = (r <= W.star_radius(th, 0.68, 0.2, 5)) & (r > 0.1)
    assert abs(int(m.sum()) - 14771) < 0.01 * 14771


def test_ode_recipes_use_the_paper_shape_parameter():
    p = W.ode(n=256)
    assert abs(p.grid.epsh - W.epsh_from_tau0(1e-10)) < 1e-15 and abs(p.k0 - 256 / 5) < 1e-15
    q = W.ode_neumann(n=256)
    g = q.boundary_rhs()[:, 0]
    assert abs(g[0] - np.sin(-q.k0)) < 1e-15 and abs(g[1] - q.k0 * np.cos(q.k0)) < 1e-12
