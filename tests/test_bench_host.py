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


def test_clock_sampler_parses_reasons_and_median():
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    cs.lines = ["0, 1500, 2070, 700, 0x8, Not Active, Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_replica_rate_single_rank():
    import bench
    v, ms = bench.replica_rate(100.0, 64, 10, 1)
    assert ms == 100.0 and abs(v - 6400.0) < 1e-9
