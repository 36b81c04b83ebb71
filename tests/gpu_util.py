"""Helpers for the GPU tests: marshal workloads problems through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev_cols(a):
    """(rows, ncols) numpy -> (ncols, rows) CUDA tensor (column-major storage)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dev())


def from_dev_cols(t):
    return t.detach().cpu().numpy().T.copy()


def setup(p, precision, k=None, seed=7, tau=1e-8, refine=-1, tau_sym=0.0):
    import paper_2308_14490_gb300 as az
    g = p.grid
    mask = torch.from_numpy(np.ascontiguousarray(p.mask.reshape(-1))).to(dev())
    bnd = None
    kernel = az.AZ_GAUSS
    if p.kind == "poisson":
        kernel = az.AZ_NEG_LAPLACE_GAUSS
        bnd = torch.from_numpy(np.ascontiguousarray(p.boundary)).to(dev())
    opts = az.make_options(precision, p.k if k is None else k, tau, tau_sym, seed, refine, p.k0)
    nrm = None
    if getattr(p, "normals", None) is not None:
        nrm = torch.from_numpy(np.ascontiguousarray(p.normals, dtype=np.float64)).to(dev())
    h = az.az_setup(az.make_grid(g.dim, g.n, g.s, g.T), mask, g.eps, kernel, bnd, p.weight, opts, normals=nrm)
    return h


def get_array(h, which, shape_cols, rows):
    import paper_2308_14490_gb300 as az
    out = torch.zeros((shape_cols, rows), dtype=torch.float64, device=dev())
    az.az_get_array(h, which, out)
    torch.cuda.synchronize()
    return from_dev_cols(out)
