"""The FP64 output of the mixed path: x = x_fp32 + correction is written as
the FP64 number nearest to the exact sum of two FP32 values, formed on the
FP32 and integer pipes.  It must equal the FP64 addition (double)a + (double)b
bit for bit, which is correctly rounded because the exact sum of two FP32
numbers is what IEEE 754 rounds once."""
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


def _cases():
    rng = np.random.default_rng(7)
    f32 = np.float32
    tiny, big = np.finfo(f32).tiny, np.finfo(f32).max
    # random pairs of every relative scale (cancellation, widely separated exponents)
    n = 1 << 20
    a = (rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))).astype(f32)
    b = (rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))).astype(f32)
    # near-cancelling pairs: b = -a (1 + small)
    c = (rng.standard_normal(n) * 1e3).astype(f32)
    d = (-c.astype(np.float64) * (1 + rng.standard_normal(n) * 1e-6)).astype(f32)
    # sums landing on powers of two, with the error pointing toward and away from zero
    p = np.exp2(rng.integers(-60, 60, 4096)).astype(f32)
    eps = (p * rng.choice([-1, 1], 4096) * np.exp2(-rng.integers(25, 60, 4096).astype(np.float64))).astype(f32)
    p2, e2 = p + eps - eps, eps                     # p2 == p: s = p exactly, e = eps
    # ties: the exact sum halfway between two FP64 numbers cannot occur for
    # nearby exponents, but can when b sits exactly at half an FP64 ulp of a
    ta = (1 + np.arange(4096) * np.exp2(-23)).astype(f32)
    tb = (ta.astype(np.float64) * np.exp2(-53)).astype(f32)
    # special values: zeros, signed zeros, subnormals, tiny and huge magnitudes
    sp = np.array([0.0, -0.0, tiny, -tiny, tiny / 8, 2.0**-75, 2.0**-76, 2.0**-74, 1.0, -1.0, big, -big, 3e38, 2.0**100],
                  dtype=f32)
    sa, sb = np.meshgrid(sp, sp)
    A = np.concatenate([a, c, p2, ta, -ta, sa.ravel()])
    B = np.concatenate([b, d, e2, tb, tb, sb.ravel()])
    return A.astype(f32), B.astype(f32)


def test_f32_sum_f64_is_the_fp64_sum(az):
    A, B = _cases()
    dev = torch.device("cuda:0")
    a = torch.from_numpy(A).to(dev)
    b = torch.from_numpy(B).to(dev)
    out = torch.empty(A.size, dtype=torch.float64, device=dev)
    az.az_debug_f32_sum_f64(a, b, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    with np.errstate(over="ignore"):
        ref = A.astype(np.float64) + B.astype(np.float64)
    same = got.view(np.int64) == ref.view(np.int64)
    bad = np.flatnonzero(~same)
    assert bad.size == 0, [(float(A[i]), float(B[i]), float(got[i]), float(ref[i])) for i in bad[:8]]


def test_f32_sum_f64_arguments(az):
    dev = torch.device("cuda:0")
    a = torch.zeros(4, dtype=torch.float32, device=dev)
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    az.az_debug_f32_sum_f64(a[:0], a[:0], out[:0])     # empty: no launch, no error
    with pytest.raises(ValueError):
        az.az_debug_f32_sum_f64(a, a, torch.zeros(4, dtype=torch.float32, device=dev))
