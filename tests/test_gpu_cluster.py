"""The cluster-resident 2D Z* chain (one 16-CTA cluster per column pair, the
grid held in distributed shared memory, enabled with AZ_SKETCH_CLUSTER=1):
against the three-pass chain (the default) and against the oracle.

Sec. 5.1 (Eq. B_pinv_2d) and Sec. 3.2.2: W = R - Z* A R, z = Z* y."""
import os

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


def _op(p):
    if p.kind == "poisson":
        return Operator(p.grid, p.mask, "poisson", p.boundary, p.weight)
    return Operator(p.grid, p.mask)


def _setup(az, p, prec, cluster, k=None, seed=5):
    os.environ["AZ_SKETCH_CLUSTER"] = "1" if cluster else "0"
    try:
        return _gu().setup(p, prec, k=k, seed=seed, refine=0 if prec == az.AZ_FP64 else 1)
    finally:
        os.environ.pop("AZ_SKETCH_CLUSTER", None)


def _arrays(az, h, p, op, k):
    gu = _gu()
    Wg = gu.get_array(h, az.AZ_ARRAY_W, k, op.N)
    Yg = gu.get_array(h, az.AZ_ARRAY_SKETCH, k, op.M + op.Mb)
    return Wg, Yg


CASES = [("disc-n32", lambda: W.config3(n=32, k=48)),
         ("star-n64", lambda: W.helmholtz(n=64, nb=4, k=40, k0=0.0)),
         ("disc-n128", lambda: W.config3(n=128, k=32)),
         ("poisson-n32", lambda: W.config4(n=32, nb=128, k=40)),
         ("poisson-n128", lambda: W.config4(n=128, nb=2048, k=24))]


def _problem(name, mk):
    p = mk()
    if name == "star-n64":
        # an approximation problem on the star (no boundary rows)
        p = W.Problem("2d-star-n64", p.grid, p.mask, p.k, [lambda q: np.cos(2 * q[:, 0]) * q[:, 1]])
    return p


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_cluster_chain_matches_three_pass_chain(az, name, mk):
    p = _problem(name, mk)
    op = _op(p)
    out = {}
    for cl in (True, False):
        h = _setup(az, p, az.AZ_FP64, cl)
        try:
            out[cl] = _arrays(az, h, p, op, p.k)
        finally:
            az.az_destroy(h)
    for a, b in zip(out[True], out[False]):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), name


@pytest.mark.parametrize("name,mk", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_cluster_sketch_columns_against_oracle(az, name, mk):
    p = _problem(name, mk)
    op = _op(p)
    R = philox.rademacher(op.N, 4, 5)
    Wref = R - op.Zstar(op.A(R))
    Yref = op.A(Wref)
    h = _setup(az, p, az.AZ_FP64, True)
    try:
        Wg, Yg = _arrays(az, h, p, op, p.k)
    finally:
        az.az_destroy(h)
    assert np.abs(Wg[:, :4] - Wref).max() <= 1e-11 * np.abs(Wref).max()
    assert np.abs(Yg[:, :4] - Yref).max() <= 1e-11 * np.abs(Yref).max()


def test_cluster_zstar_apply_and_relres_parity(az):
    gu = _gu()
    p = W.config3(n=64, k=64)
    op = _op(p)
    b = p.rhs()
    h = _setup(az, p, az.AZ_FP64, True, seed=11)
    try:
        ys = np.random.default_rng(2).standard_normal((op.M, 3))
        z = torch.zeros((3, op.N), dtype=torch.float64, device=gu.dev())
        az.az_apply_Zstar(h, gu.to_dev_cols(ys), z)
        ref = op.Zstar(ys)
        assert np.abs(gu.from_dev_cols(z) - ref).max() <= 1e-11 * np.abs(ref).max()
        x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        xg = gu.from_dev_cols(x)
    finally:
        az.az_destroy(h)
    r_o = relres(op, AZ(op, p.k, 11, 1e-8).solve(b), b)
    r_g = relres(op, xg, b)
    assert np.all(np.abs(r_g - r_o) <= 1e-10), (r_g.tolist(), r_o.tolist())
