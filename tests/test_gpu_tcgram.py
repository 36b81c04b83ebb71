"""The first Gram of the mixed factorisation, G1 = Y^T Y (the SVQB pass that
replaces the SVD of Sec. 3.2.3), by both routes the setup uses: exact FP32
products with double-float sums (route 0), and the exact split on the tensor
cores (route 1: BF16 slices of the power-of-two-scaled columns, per-CTA
slice-pair sums that are exact integers in the FP32 accumulator, FP64 fold).

The reference is exact: a product of two FP32 values is exact in FP64, and
math.fsum rounds the sum of those products once.  Route 1 drops the bits of
each scaled value below 2^-48 of its column's scale (the last slice is
rounded), so its error is at most 2^-49 max|y_a| |y_b| + 2^-49 max|y_b| |y_a|
per row, summed; an inexact tensor-core accumulation would instead show up at
about 2^-24 of the entries."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def az():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as m
    return m


def _columns(M, k, rng):
    """Columns of very different scales and shapes (k >= 7)."""
    Y = np.empty((k, M), dtype=np.float32)
    for c in range(k):
        kind = c % 7
        scale = 10.0 ** rng.uniform(-6, 6)
        if kind == 0:
            col = rng.standard_normal(M)
        elif kind == 1:
            col = np.zeros(M)                                     # a zero column
        elif kind == 2:
            col = rng.standard_normal(M) * 1e-7                   # spiky: tiny values and a few large ones
            col[rng.integers(0, M, 3)] = rng.standard_normal(3)
        elif kind == 3:
            col = np.exp2(rng.integers(-30, 30, M)).astype(np.float64) * rng.choice([-1, 1], M)   # powers of two
        elif kind == 4:
            col = 1.0 + rng.standard_normal(M) * 2.0 ** -20         # cancellation-prone: all near 1
        elif kind == 5:
            col = rng.uniform(-1, 1, M) * np.exp(rng.uniform(-20, 20, M))   # wide dynamic range
        else:
            col = rng.standard_t(2, M)                              # heavy tails
        Y[c] = (col * scale).astype(np.float32)
    return Y


def _exact(Y):
    Y64 = Y.astype(np.float64)
    k = Y.shape[0]
    G = np.empty((k, k))
    for a in range(k):
        for b in range(a, k):
            G[a, b] = G[b, a] = math.fsum((Y64[a] * Y64[b]).tolist())
    return G


def _bound(Y):
    """Per-entry error allowance of route 1 (truncation of each scaled value
    at 2^-48 of its column's scale, plus the FP64 fold and reduction)."""
    A = np.abs(Y.astype(np.float64))
    mx = A.max(axis=1)
    S = A.sum(axis=1)
    scale = np.exp2(np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 2.0)   # the column scale 2^E
    trunc = 2.0 ** -49 * (np.outer(scale, S) + np.outer(S, scale))
    return trunc + 1e-13 * (A @ A.T) + 1e-300


@pytest.mark.parametrize("M,k", [(1, 24), (1000, 24), (65536 + 37, 24), (4099, 7), (70001, 13)])
def test_gram_routes_against_exact_sums(az, M, k):
    rng = np.random.default_rng(M + k)
    Y = _columns(M, k, rng)
    dev = torch.device("cuda:0")
    ld = (M + 3) // 4 * 4                      # 16-byte column starts, a view of M rows
    Yd = torch.zeros((k, ld), dtype=torch.float32, device=dev)
    Yd[:, :M] = torch.from_numpy(Y).to(dev)
    Yd = Yd[:, :M]
    ref = _exact(Y)
    bound = _bound(Y)
    for route in (0, 1):
        G = torch.zeros((k, k), dtype=torch.float64, device=dev)
        az.az_debug_gram(Yd, G, route)
        Gh = G.cpu().numpy()
        err = np.abs(Gh - ref)
        # route 0: exact products, double-float sums (about 2^-44 of sum |y_a y_b|)
        lim = bound if route == 1 else 2.0 ** -40 * (np.abs(Y.astype(np.float64)) @ np.abs(Y.astype(np.float64)).T) + 1e-300
        bad = np.argwhere(err > lim)
        assert bad.size == 0, (route, [(int(a), int(b), float(err[a, b]), float(lim[a, b]), float(ref[a, b]))
                                       for a, b in bad[:5]])
        assert np.array_equal(Gh, Gh.T)


def test_gram_tensor_route_matches_on_plain_sketch_columns(az):
    """Gaussian columns of one scale: the two routes agree to FP64 rounding."""
    rng = np.random.default_rng(3)
    M, k = 300_000, 24
    Y = rng.standard_normal((k, M)).astype(np.float32)
    dev = torch.device("cuda:0")
    Yd = torch.from_numpy(Y).to(dev)
    Gs = []
    for route in (0, 1):
        G = torch.zeros((k, k), dtype=torch.float64, device=dev)
        az.az_debug_gram(Yd, G, route)
        Gs.append(G.cpu().numpy())
    scale = np.abs(Gs[0]).max()
    assert np.abs(Gs[0] - Gs[1]).max() <= 1e-13 * scale


def test_gram_tensor_route_limits(az):
    dev = torch.device("cuda:0")
    Y = torch.zeros((25, 64), dtype=torch.float32, device=dev)
    G = torch.zeros((25, 25), dtype=torch.float64, device=dev)
    with pytest.raises(az.AZError) as ei:
        az.az_debug_gram(Y, G, 1)          # k > 24: not the tensor-core route
    assert ei.value.status == az.AZ_ERR_ARG
    az.az_debug_gram(Y, G, 0)              # the double-float route takes it
    assert float(G.abs().max()) == 0.0
