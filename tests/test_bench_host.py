"""Host-side pieces of bench.py that need no GPU."""
import workloads as W


def test_plan_bytes_config2():
    import bench
    p = W.config2(1 << 20, 64)
    M = int(p.mask.sum())
    b = bench.plan_bytes(p.grid, M, 24, 64)
    L, N = 1 << 21, 1 << 20
    assert b == 24 * (24 * L + 4 * M) + 64 * (2 * (24 * M + 32 * L + 48 * N) + (24 * N + 16 * L + 16 * M))
    assert 20e9 < b < 30e9
