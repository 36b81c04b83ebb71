"""Benchmark of the AZ solver on the 1D-at-scale workload (one GB300 per rank).

Workload (the configuration the headline metric is quoted on): N = 2^20
Gaussian centers on [-1, 1], eps = 1/h, Omega = [-0.7, 0.3], oversampling 2,
sketch width k = 24, a batch of 64 right-hand sides cos(w x + phi) with
w ~ U[1, 40], phi ~ U[0, 2 pi) from the seed; FP32 transforms and sketch,
FP64 factor work, one FP64-residual refinement step.

One step = the whole hot path: az_refactor (index map, symbol, test matrix,
sketch, factorisation) + az_solve of the 64 right-hand sides.  value = solved
right-hand sides per second over all ranks.  Multi-GPU: independent replicas
(the solve has no exchange step); each rank times its own steps, the slowest
rank's time is used.

--impl reference times the CPU oracle (oracle/, FP64 NumPy) on the same
workload on the host cores: the full-size setup once, then one right-hand side
per step, reported as right-hand sides per second for the same step shape
(64 / (t_setup + 64 t_rhs)).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CENTERS = 1 << 20
NRHS = 64
K_SKETCH = 24
METRIC = "AZ solves/s (right-hand sides per second, setup + solve per step) at parity with the FP64 oracle"
WORKLOAD = "1d-approx N=2^20 s=2 eps=1/h Omega=[-0.7,0.3] k=24 nrhs=64 mixed(FP32 sketch/FFT, FP64 factor) +1 FP64-residual refinement"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the config 1/3/4 context legs")
    ap.add_argument("--nrhs", type=int, default=NRHS, help="right-hand sides per step (default: the workload's 64)")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="length of the serving-stream sample (Poisson arrivals, 200 req/s); 0 skips it")
    ap.add_argument("--traffic-from", default=None,
                    help="write profiles/ncu_traffic.json from an ncu DRAM-counter CSV of bench.py --lite, then exit")
    ap.add_argument("--lite", action="store_true",
                    help="timed steps only (no e2e, parity, comparator or CPU legs): the small case for profiler captures")
    return ap.parse_args()


def problem():
    import workloads as W
    return W.config2(N_CENTERS, NRHS)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- oracle legs
def host_cpu():
    """CPU model and core count of this host (lscpu), for the CPU legs."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                v = ln.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    model = v
                    break
    except Exception:
        pass
    return {"cores": os.cpu_count() or 1, "model": model or "unknown"}


def _pool_init():
    # every host core for the oracle: BLAS threads (set before numpy loads in
    # this fresh process) and scipy.fft workers (oracle.operators.WORKERS)
    n = str(os.cpu_count() or 1)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = n


def _oracle_sample(n_rhs_timed, out_q=None):
    """Run the CPU oracle on the full workload: setup once + n_rhs_timed solves."""
    import workloads as W  # noqa: F401
    from oracle.az import AZ
    from oracle.operators import Operator
    p = problem()
    t0 = time.perf_counter()
    op = Operator(p.grid, p.mask)
    az = AZ(op, K_SKETCH, 1, 1e-8)
    t_setup = time.perf_counter() - t0
    b = p.rhs()
    times = []
    for j in range(n_rhs_timed):
        t1 = time.perf_counter()
        az.solve(b[:, j % b.shape[1]:j % b.shape[1] + 1], refine=1)
        times.append(time.perf_counter() - t1)
    return t_setup, times


def _oracle_pool():
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(1, initializer=_pool_init)


def cpu_baseline_leg():
    with _oracle_pool() as pool:
        t_setup, times = pool.apply(_oracle_sample, (3,))
    t_rhs = sum(times[1:]) / len(times[1:])
    value = NRHS / (t_setup + NRHS * t_rhs)
    cpu = host_cpu()
    return {"value": value, "unit": "RHS/s", "cores": cpu["cores"], "cpu_model": cpu["model"], "kind": "oracle",
            "sample": f"full-size oracle setup ({t_setup:.2f} s) + 2 of the 64 RHS after one warm-up RHS "
                      f"({t_rhs:.3f} s each, 1 refinement); value = 64 / (t_setup + 64 t_rhs), the step shape of "
                      f"the GPU arm; scipy.fft workers and BLAS threads = {cpu['cores']} cores"}


def run_reference(args):
    """The oracle on the host cores.  One timed step = one of the workload's
    right-hand sides solved and refined (what the oracle can finish in well
    under a second); the setup (index map, symbol, sketch, factorisation) is
    timed once before the warm-up.  value = 64 / (t_setup + 64 t_rhs): the
    step shape of the GPU arm (setup + 64 right-hand sides) from the two
    measured parts; ms_per_step x steps is the timed region."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    with _oracle_pool() as pool:
        t_setup, times = pool.apply(_oracle_sample, (args.warmup + args.steps,))
    timed = times[args.warmup:]
    t_rhs = sum(timed) / len(timed)
    value = NRHS / (t_setup + NRHS * t_rhs)
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_rhs, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "step": "one right-hand side solved + 1 refinement (setup timed once before the warm-up)",
            "setup_ms": 1000.0 * t_setup,
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)", "oracle": "FP64 throughout"},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cpu["cores"], "cpu_model": cpu["model"],
                             "kind": "oracle",
                             "sample": f"setup once ({t_setup:.2f} s), then one RHS per step "
                                       f"({t_rhs:.3f} s avg over {len(timed)} steps); value = 64 / (t_setup + 64 t_rhs); "
                                       f"scipy.fft workers and BLAS threads = {cpu['cores']} cores"},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- FP64 torch comparator
def fp64_torch_comparator(p, b_dev, steps=2, warmup=1):
    """The O2 algorithm written directly in torch FP64 (torch.fft, torch.linalg.svd),
    no fusion: the 'plain FP64 GPU AZ' the metric is compared against."""
    import math
    import torch
    dev = b_dev.device
    g = p.grid
    N, s, T = g.n[0], g.s[0], g.T[0]
    L = N * s
    hL = 2 * T / L
    eps = g.eps
    mask = torch.from_numpy(p.mask).to(dev).bool()
    idx = torch.nonzero(mask).squeeze(1)
    b = b_dev.T.contiguous()  # M x nrhs

    def run():
        m = torch.arange(L, device=dev, dtype=torch.float64)
        m = torch.where(m > L / 2, m - L, m)
        gs = torch.zeros(L, dtype=torch.float64, device=dev)
        for q in range(-3, 4):
            gs += torch.exp(-(eps * (m + q * L) * hL) ** 2)
        G = torch.fft.fft(gs).real
        S = (G.reshape(s, N) ** 2).sum(0)

        def A(a):
            ah = torch.fft.fft(a, dim=0)
            return torch.fft.ifft(G[:, None] * ah.repeat(s, 1), dim=0).real[idx]

        def Z(y):
            E = torch.zeros((L, y.shape[1]), dtype=torch.float64, device=dev)
            E[idx] = y
            Y = torch.fft.fft(E, dim=0)
            ah = (G[:, None] * Y).reshape(s, N, -1).sum(0) / S[:, None]
            return torch.fft.ifft(ah, dim=0).real

        gen = torch.Generator(device=dev)
        gen.manual_seed(1)
        R = torch.randint(0, 2, (N, K_SKETCH), generator=gen, device=dev).double() * 2 - 1
        AR = A(R)
        Yk = AR - A(Z(AR))
        U, Sg, Vh = torch.linalg.svd(Yk, full_matrices=False)
        r = int((Sg > 1e-8 * Sg[0]).sum())
        gg = b - A(Z(b))
        u = Vh[:r].T @ ((U[:, :r].T @ gg) / Sg[:r, None])
        x2 = R @ u
        x = Z(b - A(x2)) + x2
        return x, A

    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        x, A = run()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    rel = (torch.linalg.norm(A(x) - b, dim=0) / torch.linalg.norm(b, dim=0)).cpu().numpy()
    return {"value": NRHS / (ms / 1000.0), "unit": "RHS/s", "ms_per_step": ms, "steps": steps,
            "what": "same step (setup + 64 RHS) written in plain torch FP64 (torch.fft + torch.linalg.svd), no refinement"}, rel


# --------------------------------------------------------------------------- serving sample
def _latency(ms):
    ms = sorted(ms)
    return {"p50": ms[len(ms) // 2], "p99": ms[min(len(ms) - 1, int(0.99 * len(ms)))], "max": ms[-1]}


def config1_leg(reps=100):
    """Config 1 (1D, N = 256, Omega = [-0.5, 0.5], k = 20, FP64 only): latency of
    one whole AZ call -- az_refactor (index map, symbol, sketch, factorisation)
    and az_solve of its one right-hand side -- on the host clock, synchronised."""
    import numpy as np
    import torch
    import paper_2308_14490_gb300 as az
    import workloads as W
    dev = torch.device("cuda", 0)
    p = W.config1()
    g = p.grid
    mask = torch.from_numpy(p.mask).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(p.rhs().T)).to(dev)
    x = torch.zeros((1, g.N), dtype=torch.float64, device=dev)
    opts = az.make_options(az.AZ_FP64, p.k, 1e-8, 0.0, 7, 0)
    h = az.az_setup(az.make_grid(1, g.n, g.s, g.T), mask, g.eps, options=opts)
    ms = []
    for i in range(reps + 5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        az.az_refactor(h, 7, None)
        az.az_solve(h, b, x)
        torch.cuda.synchronize(dev)
        if i >= 5:
            ms.append(1000.0 * (time.perf_counter() - t0))
    rr = az.az_solve(h, b, x, relres=True)
    az.az_destroy(h)
    return {"what": "1D N=256 Omega=[-0.5,0.5] k=20 FP64: az_refactor + az_solve (1 RHS), host clock, synchronised",
            "latency_ms": _latency(ms), "calls": reps, "relres": rr[0]}


def config_2d_leg(name, nrhs=64):
    """Configs 3 and 4 at full size, at the sketch width the adaptive setup
    settles on (disc n = 256: k = 4096; star Poisson n = 128: k = 2048):
    setup time, solve throughput of a batch of 64 right-hand sides (the
    workload's function repeated), and the mixed path against the FP64 path
    (relres; config 4 also the maximum error of u on the 1024 x 1024 test grid
    inside the star, s_test = 8)."""
    import numpy as np
    import torch
    import paper_2308_14490_gb300 as az
    import workloads as W
    dev = torch.device("cuda", 0)
    if name == "config3":
        p = W.config3(n=256, k=4096)
    else:
        p = W.config4(n=128, nb=2048, k=2048)
    g = p.grid
    mask = torch.from_numpy(np.ascontiguousarray(p.mask.reshape(-1))).to(dev)
    kernel, bnd = az.AZ_GAUSS, None
    if p.kind == "poisson":
        kernel = az.AZ_NEG_LAPLACE_GAUSS
        bnd = torch.from_numpy(np.ascontiguousarray(p.boundary)).to(dev)
        f = torch.from_numpy(np.ascontiguousarray(np.repeat(p.rhs().T, nrhs, 0))).to(dev)
        gb = torch.from_numpy(np.ascontiguousarray(np.repeat(p.boundary_rhs().T, nrhs, 0))).to(dev)
    else:
        b = torch.from_numpy(np.ascontiguousarray(np.repeat(p.rhs().T, nrhs, 0))).to(dev)
    out = {"N": g.N, "k": p.k}
    xs = {}
    for prec, tag in ((az.AZ_FP64, "fp64"), (az.AZ_MIXED, "mixed")):
        opts = az.make_options(prec, p.k, 1e-8, 0.0, 13, -1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = az.az_setup(az.make_grid(2, g.n, g.s, g.T), mask, g.eps, kernel, bnd, p.weight, opts)
        info = az.az_get_info(h)
        setup_ms = 1000.0 * (time.perf_counter() - t0)
        x = torch.zeros((nrhs, g.N), dtype=torch.float64, device=dev)

        def solve(rel=False):
            if p.kind == "poisson":
                return az.az_collocate(h, f, gb, x, relres=rel)
            return az.az_solve(h, b, x, relres=rel)

        solve()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            solve()
        e1.record()
        torch.cuda.synchronize(dev)
        solve_ms = e0.elapsed_time(e1) / 3
        rr = solve(True)
        xs[tag] = x[:1].clone()
        ent = {"setup_ms": round(setup_ms, 1), "rank": info["rank"], "M": info["M"], "Mb": info["Mb"],
               "solve_ms_per_batch": round(solve_ms, 3), "solve_rhs_per_s": nrhs / (solve_ms / 1000.0),
               "relres": rr[0], "device_bytes": info["device_bytes"]}
        if p.kind == "poisson":
            st = 8
            vals = torch.zeros((1, g.N * st * st), dtype=torch.float64, device=dev)
            az.az_evaluate(h, x[:1], st, vals)
            gf = W.Grid(2, g.n, (st, st), g.T, g.epsh)
            inside = W.star_mask(gf).reshape(-1).astype(bool)
            X, Y = np.meshgrid(W.grid_coords(gf, 0), W.grid_coords(gf, 1), indexing="ij")
            u = p.exact[0](np.stack([X.reshape(-1), Y.reshape(-1)], 1))
            v = vals.cpu().numpy()[0]
            ent["max_error_1024"] = float(np.abs(v - u)[inside].max())
            xs[tag + "_vals"] = v[inside]
        az.az_destroy(h)
        torch.cuda.empty_cache()
        out[tag] = ent
    # the oracle's relres of the same problem (same R, k, tau), stored by
    # tests/golden/make_fullsize_relres.py: FP64 (no refinement) and mixed (one
    # refinement) against the oracle with the same refinement count
    try:
        gold = json.load(open(os.path.join(ROOT, "tests", "golden", "fullsize_relres.json")))[name]
        if gold["k"] == p.k:
            out["oracle_relres_refine0"] = gold["relres_refine0"]
            out["oracle_relres_refine1"] = gold["relres_refine1"]
            out["gap_fp64_vs_oracle"] = abs(out["fp64"]["relres"] - gold["relres_refine0"])
            out["gap_mixed_vs_oracle"] = abs(out["mixed"]["relres"] - gold["relres_refine1"])
    except Exception:
        pass
    out["relres_gap_mixed_vs_fp64"] = abs(out["mixed"]["relres"] - out["fp64"]["relres"])
    if p.kind == "poisson":
        out["max_abs_diff_u_mixed_vs_fp64_1024"] = float(np.abs(xs["mixed_vals"] - xs["fp64_vals"]).max())
    out["what"] = (f"{p.name}: az_setup wall time, az_solve/az_collocate of {nrhs} copies of the workload RHS "
                   "(CUDA events, mean of 3 batches), relres of the first; mixed = FP64 sketch and factors, "
                   "FP32 solve transforms, 1 FP64-residual refinement")
    return out


def cluster_leg():
    """The FP64 Z* chain of the config-4 sketch (n = 128, L = 256^2, k = 2048,
    1024 column pairs) as three passes through device memory (the default)
    and as the cluster-resident kernel (AZ_SKETCH_CLUSTER=1: one 16-CTA
    cluster per pair, the grid in distributed shared memory): device time of
    the chain from CUDA events around its launches during az_setup."""
    import numpy as np
    import torch
    import paper_2308_14490_gb300 as az
    import workloads as W
    dev = torch.device("cuda", 0)
    p = W.config4(n=128, nb=2048, k=2048)
    g = p.grid
    mask = torch.from_numpy(np.ascontiguousarray(p.mask.reshape(-1))).to(dev)
    bnd = torch.from_numpy(np.ascontiguousarray(p.boundary)).to(dev)
    out = {}
    for tag, env in (("three_pass", "0"), ("cluster", "1")):
        os.environ["AZ_SKETCH_CLUSTER"] = env
        try:
            opts = az.make_options(az.AZ_FP64, p.k, 1e-8, 0.0, 13, 0)
            az.az_profile_begin()
            h = az.az_setup(az.make_grid(2, g.n, g.s, g.T), mask, g.eps, az.AZ_NEG_LAPLACE_GAUSS, bnd, p.weight, opts)
            prof = az.az_profile_end()
            az.az_destroy(h)
        finally:
            os.environ.pop("AZ_SKETCH_CLUSTER", None)
        keys = [k for k in prof if k.startswith(("colfwd_", "rowfold_", "colinv_", "zstar_cluster"))]
        ms = sum(prof[k]["ms"] for k in keys)
        out[tag] = {"ms": round(ms, 3), "us_per_pair": round(1000.0 * ms / (p.k // 2), 2), "kernels": sorted(keys)}
    # FP64 flops per pair: forward 2D FFT of the L-grid, inverse of the N-grid (5 n log2 n each), fold
    L2, N2 = (2 * g.n[0]) ** 2, g.n[0] ** 2
    flop = 5 * L2 * np.log2(L2) + 5 * N2 * np.log2(N2) + 8 * L2
    for tag in out:
        out[tag]["fp64_tflops"] = round(flop * (p.k // 2) / (out[tag]["ms"] / 1000.0) / 1e12, 3)
    out["what"] = ("config-4 sketch Z* chain (FP64, 1024 column pairs): three passes vs the cluster-resident kernel; "
                   "FP64-arithmetic bound (peak about 1.26 TFLOP/s on this GPU)")
    return out


def fp64_step_leg(h_grid, mask, b_dev, x_dev, stream, steps=5):
    """The library's own all-FP64 config-2 step (az_refactor + az_solve of 64 RHS)."""
    import torch
    import paper_2308_14490_gb300 as az
    g = problem().grid
    o64 = az.make_options(az.AZ_FP64, K_SKETCH, 1e-8, 0.0, 1, 0)
    h = az.az_setup(h_grid, mask, g.eps, options=o64)
    for i in range(2):
        az.az_refactor(h, 1 + i, stream)
        az.az_solve(h, b_dev, x_dev, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        az.az_refactor(h, 1 + (i % 2), stream)
        az.az_solve(h, b_dev, x_dev, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    az.az_destroy(h)
    return {"value": NRHS / (ms / 1000.0), "unit": "RHS/s", "ms_per_step": ms, "steps": steps,
            "what": "same step, library all-FP64 path (FP64 sketch, transforms, factor and solve, no refinement)"}


def serving_leg(seconds):
    """The mixed request stream: Poisson arrivals at 200/s of 1D / 2D approximations
    and 2D Poisson collocations drawn from a seeded pool of 32 setups, 1..32 RHS
    each, continuous batching over 4 streams with CUDA-graph replay.  Three runs of
    the same stream: mixed precision from a cold start (each setup built on its
    first request), then mixed and all-FP64 with the pool built beforehand."""
    import paper_2308_14490_gb300 as az
    import paper_2308_14490_gb300.serving as S
    pool = S.setup_pool(230814490, 32)
    reqs = S.poisson_stream(230814490, 200.0, seconds, pool)
    cold_s = min(seconds, 20.0)
    reqs_cold = [r for r in reqs if r.arrival <= cold_s]
    out = {}
    for name, prec, warm in (("mixed_cold", az.AZ_MIXED, False), ("mixed_warm", az.AZ_MIXED, True),
                             ("fp64_warm", az.AZ_FP64, True)):
        srv = S.Server(64 << 30, nslots=4, precision=prec)
        warm_ms = srv.warm(pool) if warm else 0.0
        fresh = [S.Request(r.rid, r.arrival, r.spec, r.nrhs, r.seed) for r in (reqs if warm else reqs_cold)]
        res = srv.run(fresh, realtime=True)
        if warm:
            res["warm_up_ms"] = warm_ms
            # capacity: the same requests all queued at once (closed loop, no
            # arrival gaps); only the throughput of this run is meaningful
            again = [S.Request(r.rid, r.arrival, r.spec, r.nrhs, r.seed) for r in reqs]
            cap = srv.run(again, realtime=False)
            res["capacity_solves_per_s"] = cap["solves_per_s"]
        srv.close()
        out[name] = res
    out["stream"] = (f"{len(reqs)} requests over {seconds:.0f} s (Poisson 200/s; the cold run takes the first "
                     f"{cold_s:.0f} s, {len(reqs_cold)} requests), pool of 32 setups; 2D setups at k = 64 (below their "
                     "rank: parity with the oracle at that width, not the resolved residual); each request's result "
                     "equals its result alone (even-aligned batch columns)")
    return out


# --------------------------------------------------------------------------- replicas
def replica_rate(local_ms: float, nrhs: int, steps: int, world: int, dist=None, device=None):
    """Whole-job rate of independent replicas: the slowest rank's time bounds the
    job; every rank solved nrhs * steps right-hand sides."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return world * nrhs * steps / (total_ms / 1000.0), total_ms


# --------------------------------------------------------------------------- our arm
def csrc_digest():
    """SHA-1 over the CUDA sources: DRAM counters taken on other sources are stale."""
    import hashlib
    d = os.path.join(ROOT, "paper_2308_14490_gb300", "csrc")
    h = hashlib.sha1()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def load_traffic():
    """Per-kernel DRAM bytes from one ncu pass, or {} when the kernels changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        t = json.load(open(path))
    except Exception:
        return {}
    if t.get("csrc_sha1") != csrc_digest():
        return {}
    return t.get("kernels", {})


# ncu kernel names -> the library's kernel-class labels (ProfScope names)
TRAFFIC_LABELS = [
    (r"^k_colfwd_r<float, 0", "colfwd_gather_f32"), (r"^k_colfwd_r<float, 1", "colfwd_sketch_f32"),
    (r"^k_rowfold_r<float", "rowfold_f32"), (r"^k_colinv_r<float", "colinv_f32"),
    (r"^k_stencil_rows<float", "stencil_rows_f32"), (r"^k_resid_df", "resid_df"),
    (r"^k_update_x", "update_x"), (r"^k_tc_tsgram", "proj_tc"), (r"^k_tc_gram_oz", "gram_oz"),
    (r"^k_gram_reduce", "gram_reduce"),
    (r"^k_gram_partial", "gram_df32"), (r"^k_tsprod_df", "tsprod_df32"), (r"^k_tsprod<", "tsprod"),
    (r"^k_small_mm", "small_mm"), (r"^k_factor1", "factor1"), (r"^k_factor2", "factor2"),
    (r"^k_count|^k_scan_blocks|^k_scatter", "compact"), (r"^k_taps", "taps"),
    (r"^k_symbol_closed_1d|^k_fold_S|^k_max_abs|^k_H", "symbol"), (r"^k_philox_bits", "philox_bits"),
]


def traffic_from_csv(csv_path, steps=1):
    """profiles/ncu_traffic.json from the CSV of
    ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
        --csv --log-file <csv> python bench.py --lite --steps <steps> --warmup 3
    (the launches of the last `steps` timed steps are the run's final launches)."""
    import csv
    import re
    rows = [r for r in csv.reader(open(csv_path)) if len(r) > 10]
    head = rows[0]
    ci, cn, cm, cv = head.index("ID"), head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Value")
    per = {}
    for r in rows[1:]:
        ent = per.setdefault(int(r[ci]), {"name": r[cn]})
        ent[r[cm]] = float(r[cv].replace(",", ""))
    ids = sorted(per)
    # the timed steps' launches: the step's launch count from the run's last az_refactor (k_count)
    starts = [i for i in ids if "k_count(" in per[i]["name"]]
    first = starts[-steps] if len(starts) >= steps else ids[0]
    kern = {}
    for i in ids:
        if i < first:
            continue
        nm = re.sub(r"^void\s+", "", per[i]["name"]).replace("az::", "").replace("<unnamed>::", "")
        lab = next((l for rx, l in TRAFFIC_LABELS if re.search(rx, nm)), nm.split("<")[0])
        e = kern.setdefault(lab, {"dram_bytes_per_step": 0.0, "launches_per_step": 0, "kernels": []})
        e["dram_bytes_per_step"] += (per[i].get("dram__bytes_read.sum", 0) + per[i].get("dram__bytes_write.sum", 0)) / steps
        e["launches_per_step"] += 1
        short = nm.split("(")[0]
        if short not in e["kernels"]:
            e["kernels"].append(short)
    for e in kern.values():
        e["launches_per_step"] //= steps
        e["dram_bytes_per_step"] = int(e["dram_bytes_per_step"])
    out = {"what": "DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per kernel label over the timed step of "
                   "bench.py --lite (1D N=2^20, k=24, 64 RHS, mixed); a projection label includes its partial-sum "
                   "reduction launch",
           "command": "python -c \"import __graft_entry__ as g; g.build()\" && python bench.py --lite --steps 1 --warmup 3 "
                      "&& ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                      "--clock-control none --csv --log-file traffic_lite.csv python bench.py --lite --steps 1 --warmup 3 "
                      "&& python bench.py --traffic-from traffic_lite.csv",
           "csrc_sha1": csrc_digest(), "source": "ncu DRAM counters, timed step of bench.py --lite", "kernels": kern}
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return path


def plan_bytes(g, M, k, nrhs):
    """Pass-plan byte model of one step (sketch of width k, then the mixed
    refined solve of nrhs right-hand sides) on grid g with M kept points."""
    Lg, Ng = g.Ltot, g.N
    return k * (24 * Lg + 4 * M) + nrhs * (2 * (24 * M + 32 * Lg + 48 * Ng) + (24 * Ng + 16 * Lg + 16 * M))


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as az

    global NRHS
    NRHS = args.nrhs
    p = problem()
    g = p.grid
    b_host = np.ascontiguousarray(p.rhs()[:, :NRHS].T)  # (nrhs, M)
    M = b_host.shape[1]
    b_pin = torch.from_numpy(b_host).pin_memory()
    b_dev = b_pin.to(dev)
    x_dev = torch.zeros((NRHS, g.N), dtype=torch.float64, device=dev)
    x_pin = torch.zeros((NRHS, g.N), dtype=torch.float64).pin_memory()
    mask = torch.from_numpy(p.mask).to(dev)
    stream = torch.cuda.current_stream(dev)
    opts = az.make_options(az.AZ_MIXED, K_SKETCH, 1e-8, 0.0, 1, 1)
    h = az.az_setup(az.make_grid(1, g.n, g.s, g.T), mask, g.eps, options=opts)

    def step(i):
        az.az_refactor(h, 1 + (i % 2), stream)
        az.az_solve(h, b_dev, x_dev, stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for i in range(args.warmup):
        step(i)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    n0 = az.az_launch_count()
    barrier()
    evs[0].record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    launches = az.az_launch_count() - n0
    barrier()
    clk = clocks.stop()

    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    value, total_ms = replica_rate(evs[0].elapsed_time(evs[-1]), NRHS, args.steps, world, dist, dev)
    if args.lite:
        if rank == 0:
            print(json.dumps({"lite": True, "value": value, "ms_per_step": total_ms / args.steps,
                              "gpu_launches": int(launches)}), flush=True)
        az.az_destroy(h)
        return

    # per-kernel device time of the same steps (CUDA events around every
    # launch), taken after the timed region so that the events do not weigh
    # on the headline
    az.az_profile_begin()
    for i in range(min(args.steps, 10)):
        step(args.warmup + args.steps + i)
    torch.cuda.synchronize(dev)
    prof = az.az_profile_end()

    # end-to-end through the public API with host buffers: every step copies its
    # b from pinned host memory and reads its x back.  Copies run on their own
    # streams, double-buffered, so step i's compute overlaps the H2D of step
    # i+1 and the D2H of step i-1 (the pipeline fill and drain are timed too).
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    b_bufs = [b_dev, torch.empty_like(b_dev)]
    x_bufs = [x_dev, torch.empty_like(x_dev)]
    x_pins = [x_pin, torch.empty_like(x_pin).pin_memory()]
    ev = lambda: torch.cuda.Event()
    b_ready, b_free, x_done, x_free = [ev(), ev()], [ev(), ev()], [ev(), ev()], [ev(), ev()]
    e_evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    e_evs[0].record(stream)
    h2d.wait_event(e_evs[0])
    for i in range(args.steps):
        j = i % 2
        if i >= 2:
            h2d.wait_event(b_free[j])
        with torch.cuda.stream(h2d):
            b_bufs[j].copy_(b_pin, non_blocking=True)
        b_ready[j].record(h2d)
        stream.wait_event(b_ready[j])
        if i >= 2:
            stream.wait_event(x_free[j])
        az.az_refactor(h, 1 + (i % 2), stream)
        az.az_solve(h, b_bufs[j], x_bufs[j], stream)
        b_free[j].record(stream)
        x_done[j].record(stream)
        d2h.wait_event(x_done[j])
        with torch.cuda.stream(d2h):
            x_pins[j].copy_(x_bufs[j], non_blocking=True)
        x_free[j].record(d2h)
    for j in range(min(2, args.steps)):
        stream.wait_event(x_free[j])
    e_evs[1].record(stream)
    torch.cuda.synchronize(dev)
    e_val, _ = replica_rate(e_evs[0].elapsed_time(e_evs[1]), NRHS, args.steps, world, dist, dev)
    e2e = {"value": e_val, "unit": "RHS/s",
           "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(x_pin.numel() * 8),
           "copies": "pinned host buffers; H2D and D2H on their own streams, double-buffered against the compute"}
    # the same two copies alone on this machine (both directions at once, no
    # compute): whether the end-to-end rate is bound by the link or the step
    c_evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ncopy = 3
    torch.cuda.synchronize(dev)
    c_evs[0].record(h2d)
    d2h.wait_stream(h2d)
    for i in range(ncopy):
        with torch.cuda.stream(h2d):
            b_bufs[1].copy_(b_pin, non_blocking=True)
        with torch.cuda.stream(d2h):
            x_pins[1].copy_(x_bufs[1], non_blocking=True)
    h2d.wait_stream(d2h)
    c_evs[1].record(h2d)
    torch.cuda.synchronize(dev)
    copy_ms = c_evs[0].elapsed_time(c_evs[1]) / ncopy
    e2e["copies_only_ms_per_step"] = round(copy_ms, 3)
    e2e["compute_ms_per_step"] = round(total_ms / args.steps, 3)
    e2e["bound_by"] = "copies" if copy_ms > total_ms / args.steps else "compute"

    # parity: relres of the mixed result vs the library's all-FP64 path on the same batch
    rr_mixed = az.az_solve(h, b_dev, x_dev, stream, relres=True)
    o64 = az.make_options(az.AZ_FP64, K_SKETCH, 1e-8, 0.0, 1, 0)
    h64 = az.az_setup(az.make_grid(1, g.n, g.s, g.T), mask, g.eps, options=o64)
    x64 = torch.zeros_like(x_dev)
    rr64 = az.az_solve(h64, b_dev, x64, stream, relres=True)
    info = az.az_get_info(h)
    az.az_destroy(h64)

    # roofline of the dominant kernel.  In the timed steps the refactor's sketch
    # runs on the setup's own stream beside the solve's first Z* pass, so a
    # launch's event-to-event time there includes sharing the GPU; the
    # per-kernel durations of the roofline come from the same steps run again
    # with the refactor finished before the solve starts (each launch alone).
    az.az_profile_begin()
    for i in range(3):
        az.az_refactor(h, 1 + (i % 2), stream)
        torch.cuda.synchronize(dev)
        az.az_solve(h, b_dev, x_dev, stream)
    torch.cuda.synchronize(dev)
    prof_iso = az.az_profile_end()
    dom, ent = max(prof_iso.items(), key=lambda kv: kv[1]["ms"])
    ent_t = prof.get(dom, {"ms": 0.0, "launches": 1})
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = ent["bytes"] / (ent["ms"] / 1000.0) / 1e9
    tr = load_traffic().get(dom)
    share = {k: round(v["ms"] / sum(e["ms"] for e in prof.values()), 4) for k, v in
             sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_source": peak_src,
                "traffic": (tr["dram_bytes_per_step"] / tr["launches_per_step"]) if tr else None,
                "traffic_source": "profiles/ncu_traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass over the timed step of bench.py --lite)" if tr else None,
                "algorithmic_bytes_per_launch": ent["bytes"] / max(1, ent["launches"]),
                "avg_launch_ms": ent["ms"] / max(1, ent["launches"]),
                "avg_launch_ms_in_timed_steps": ent_t["ms"] / max(1, ent_t["launches"]),
                "durations": "CUDA events around each launch on its stream, 3 steps with the refactor finished before "
                             "the solve; time_share and avg_launch_ms_in_timed_steps from a profiled repeat of the "
                             "timed steps (refactor overlapping the solve)",
                "time_share": share}

    # whole step against the pass-plan byte model fixed in advance for this
    # workload: sketch k (24 L + 4 M) plus, per right-hand side of the mixed
    # refined solve, (24 M + 32 L + 48 N) twice and the FP64 residual
    # (24 N + 16 L + 16 M); and against the DRAM bytes ncu measured per step
    plan = plan_bytes(g, M, K_SKETCH, NRHS)
    step_s = total_ms / args.steps / 1000.0
    measured = sum(v["dram_bytes_per_step"] for v in load_traffic().values()) or None
    step_roofline = {"bound": "hbm", "plan_bytes_per_step": int(plan), "achieved": round(plan / step_s / 1e9, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(plan / step_s / 1e9 / hbm, 4),
                     "dram_bytes_per_step": measured,
                     "dram_frac": round(measured / step_s / 1e9 / hbm, 4) if measured else None}

    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": g.N, "M": int(M), "k": K_SKETCH, "nrhs": NRHS,
                       "rank_kept": info["rank"], "l2": "no flush: inputs (b 537 MB) and per-step working set (>1 GB) exceed L2",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": sorted(per)[len(per) // 2], "p99": sorted(per)[min(len(per) - 1, int(0.99 * len(per)))],
                           "max": max(per)},
            "parity": {"relres_max_mixed": max(rr_mixed), "relres_max_fp64": max(rr64),
                       "max_gap_mixed_vs_fp64": max(abs(a - c) for a, c in zip(rr_mixed, rr64)), "tol": 1e-8},
            "roofline": roofline, "step_roofline": step_roofline, "gpu_launches": int(launches), "clocks": clk,
            "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_comparator:
        try:
            comp, rel = fp64_torch_comparator(p, b_dev)
            comp["relres_max"] = float(rel.max())
            line["fp64_gpu_torch"] = comp
        except Exception as ex:  # the comparator is context, never the headline
            line["fp64_gpu_torch"] = {"error": str(ex)[:200]}
        try:
            line["fp64_library_step"] = fp64_step_leg(az.make_grid(1, g.n, g.s, g.T), mask, b_dev, x_dev, stream)
        except Exception as ex:
            line["fp64_library_step"] = {"error": str(ex)[:200]}
    az.az_destroy(h)
    if rank == 0 and world == 1 and args.serving_seconds > 0:
        line["serving"] = serving_leg(args.serving_seconds)
    if rank == 0 and world == 1 and not args.no_context:
        for nm, fn in (("config1", config1_leg), ("config3", lambda: config_2d_leg("config3")),
                       ("config4", lambda: config_2d_leg("config4")), ("cluster_zstar", cluster_leg)):
            try:
                line[nm] = fn()
            except Exception as ex:  # context, never the headline
                line[nm] = {"error": str(ex)[:300]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.traffic_from:
        print(traffic_from_csv(a.traffic_from))
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
