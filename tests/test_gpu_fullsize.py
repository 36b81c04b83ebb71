"""Configs 3 and 4 at their full sizes and sketch widths (2D disc n = 256,
k = 4096; Poisson on the star, n = 128, 2048 boundary points, k = 2048).

End-to-end parity: the relative residual of the workload's right-hand side
against the oracle's Algorithm 1 with the same R (seed 13), k, tau = 1e-8 and
refinement count -- FP64 within 1e-10, mixed within 1e-8 -- and the FP64 rank
equal to the oracle's.  The oracle values are in tests/golden/fullsize_relres.json,
written by tests/golden/make_fullsize_relres.py (CPU, several minutes).  Sampled
sketch columns W_j = R_j - Z* A R_j and Y_j = A W_j are compared entry by entry
with the oracle, which computes a few columns in seconds."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import philox
from oracle.az import relres
from oracle.operators import Operator

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 13
NCHECK = 3


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


def _rhs(p, op):
    if p.kind == "poisson":
        return np.concatenate([p.rhs() / (2 * op.eps ** 2), p.weight * p.boundary_rhs()])
    return p.rhs()


def _sample_and_solve(az, p, op, prec):
    gu = _gu()
    h = gu.setup(p, prec, seed=SEED)
    try:
        Wg = gu.get_array(h, az.AZ_ARRAY_W, p.k, op.N)[:, :NCHECK]
        Yg = gu.get_array(h, az.AZ_ARRAY_SKETCH, p.k, op.M + op.Mb)[:, :NCHECK]
        b = _rhs(p, op)
        x = torch.zeros((b.shape[1], op.N), dtype=torch.float64, device=gu.dev())
        az.az_solve(h, gu.to_dev_cols(b), x)
        r = relres(op, gu.from_dev_cols(x), b)
        info = az.az_get_info(h)
    finally:
        az.az_destroy(h)
        torch.cuda.empty_cache()
    return Wg, Yg, r, info


GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_relres.json")))


def _problem(name):
    g = GOLDEN[name]
    if name == "config3":
        return W.config3(n=256, k=g["k"])
    return W.config4(n=128, nb=2048, k=g["k"])


@pytest.mark.parametrize("name", ["config3", "config4"])
def test_fullsize_relres_parity(az, name):
    gold = GOLDEN[name]
    p = _problem(name)
    op = _op(p)
    assert (op.N, op.M, op.Mb) == (gold["N"], gold["M"], gold["Mb"])
    for prec, refine, key, tol in ((az.AZ_FP64, 0, "relres_refine0", 1e-10), (az.AZ_MIXED, 1, "relres_refine1", 1e-8)):
        gu = _gu()
        h = gu.setup(p, prec, seed=SEED, refine=refine)
        try:
            info = az.az_get_info(h)
            assert info["k"] == gold["k"]
            if prec == az.AZ_FP64:
                assert info["rank"] == gold["rank"]
            b = _rhs(p, op)
            x = torch.zeros((1, op.N), dtype=torch.float64, device=gu.dev())
            rr = az.az_solve(h, gu.to_dev_cols(b), x, relres=True)
        finally:
            az.az_destroy(h)
            torch.cuda.empty_cache()
        print(name, prec, rr[0], gold[key], rr[0] - gold[key])
        assert abs(rr[0] - gold[key]) <= tol, (name, prec, rr[0], gold[key])


@pytest.mark.parametrize("name", ["config3", "config4"])
def test_fullsize_sketch_columns_and_residuals(az, name):
    p = W.config3(n=256, k=1024) if name == "config3" else W.config4()
    op = _op(p)
    R = philox.rademacher(op.N, NCHECK, SEED)
    Wref = R - op.Zstar(op.A(R))
    Yref = op.A(Wref)
    # (2D mixed setups sketch in FP64, so both precisions meet the FP64 bound)
    for prec in (az.AZ_FP64, az.AZ_MIXED):
        Wg, Yg, r, info = _sample_and_solve(az, p, op, prec)
        assert info["k"] == p.k and info["rank"] >= 1
        assert np.abs(Wg - Wref).max() <= 1e-11 * np.abs(Wref).max()
        assert np.abs(Yg - Yref).max() <= 1e-11 * np.abs(Yref).max()
