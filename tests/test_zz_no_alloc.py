"""The allocation-free Rademacher entry point gives the same matrix as the
allocating one.

az_rademacher_noalloc exists for callers that cannot allocate device memory
(for example when a caching allocator already holds the free HBM, or when
cudaMalloc/cudaFree would synchronise a latency-critical path).  This file is
collected last on purpose, and must also pass when run on its own.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as az
    return az


def test_noalloc_rademacher_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    az = _lib()
    dev = torch.device("cuda:0")
    # two calls in a row on the shared scratch, different shapes and seeds
    for (N, k, seed) in [(100003, 24, 7), (4096, 5, 2 ** 40 + 3)]:
        R_ref = torch.zeros((k, N), dtype=torch.float64, device=dev)
        R_new = torch.full((k, N), 9.0, dtype=torch.float64, device=dev)
        az.az_rademacher(N, k, seed, R_ref)
        az.az_rademacher_noalloc(N, k, seed, R_new)
        torch.cuda.synchronize()
        assert torch.equal(R_ref, R_new)
        assert set(np.unique(R_new.cpu().numpy())) == {-1.0, 1.0}


def test_noalloc_matches_the_oracle_rademacher_on_a_user_stream():
    """Two calls back to back on one non-default stream, different shapes and
    seeds, no synchronisation between them: each output equals the oracle's
    Philox4x32-10 Rademacher matrix (the published generator, written on the
    CPU) and the allocating entry point's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.philox import rademacher
    az = _lib()
    dev = torch.device("cuda:0")
    cases = [(70001, 9, 11), (3000, 17, 2 ** 33 + 5)]
    st = torch.cuda.Stream(dev)
    outs = [torch.full((k, N), 9.0, dtype=torch.float64, device=dev) for (N, k, _) in cases]
    torch.cuda.synchronize()
    for (N, k, seed), R in zip(cases, outs):
        az.az_rademacher_noalloc(N, k, seed, R, stream=st)
    st.synchronize()
    for (N, k, seed), R in zip(cases, outs):
        ref = rademacher(N, k, seed)                  # (N, k) from the oracle
        assert np.array_equal(R.cpu().numpy().T, ref)
        R_alloc = torch.zeros((k, N), dtype=torch.float64, device=dev)
        az.az_rademacher(N, k, seed, R_alloc)
        torch.cuda.synchronize()
        assert torch.equal(R_alloc, R)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    az = _lib()
    R = torch.zeros((1, 8), dtype=torch.float64, device="cuda:0")
    with pytest.raises(az.AZError) as ei:
        az.az_rademacher_noalloc(1 << 26, 1, 1, R)   # rejected on the host, before any launch
    assert ei.value.status == az.AZ_ERR_ARG
    assert "exceeds the fixed scratch" in str(ei.value)
    with pytest.raises(az.AZError) as ei:
        az.az_rademacher_noalloc(8, 70000, 1, R)     # k above the grid's 65535 rows, within the scratch
    assert ei.value.status == az.AZ_ERR_ARG
    assert "65535" in str(ei.value)
