"""Continuous-batching request loop for AZ solves (approximation and collocation).

* Setups (grid, domain, kernel) are created on first use and kept resident
  on the device -- symbols, index maps, sketch factors and workspace -- so
  repeated right-hand sides only pay for az_solve / az_collocate.
* Admission by device footprint: before a new setup is built its bytes are
  estimated with az_query_footprint; least-recently-used idle setups are
  evicted to fit the budget, and a setup that cannot fit is rejected
  (AZ_ERR_ADMISSION semantics; the request is counted as rejected).
* Continuous batching: queued requests for the same setup are merged into
  one solve (their right-hand-side columns concatenated, padded to a bucket of
  2/4/8/16/32/64 columns) and dispatched to a free slot as soon as one frees
  up; each slot is its own CUDA stream, so batches of different setups overlap
  on the device while new requests keep arriving.
* Each (setup, bucket) solve is captured once into a CUDA graph and replayed.
  A bucket's first solve runs eagerly; its capture (which waits for the whole
  device) is deferred to a moment when no request is queued or running.
* Optional warm start: ``Server.warm`` builds a known pool of setups (and
  captures their graphs) before requests arrive, so that the stream measures
  steady-state serving; a cold run builds each setup on its first request.
* ``precision`` selects the mixed (FP32 sketch and transforms, FP64 factor and
  residual) or the all-FP64 path for every setup of the server.

Right-hand sides are generated on the device from each request's seeded
parameters (workload inputs, not solver arithmetic).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (AZ_ERR_ADMISSION, AZ_FP64, AZ_GAUSS, AZ_MIXED, AZ_NEG_LAPLACE_GAUSS, AZError, az_collocate, az_destroy,
               az_get_info, az_query_footprint, az_setup, az_solve, make_grid, make_options)

BUCKETS = (2, 4, 8, 16, 32, 64)


@dataclass
class SetupSpec:
    """One problem: dim, centers per dim, oversampling, half-widths, domain."""
    key: tuple
    dim: int
    n: tuple
    s: tuple
    T: tuple
    kind: str                  # "approx" | "poisson"
    mask_fn: object            # callable(grid coordinate arrays) -> bool mask
    boundary: np.ndarray | None = None
    weight: float = 10.0
    k: int = 24
    epsh: float = 1.0


@dataclass
class Request:
    rid: int
    arrival: float             # seconds since the start of the run
    spec: SetupSpec
    nrhs: int
    seed: int
    t_done: float = -1.0
    rejected: bool = False


class _Setup:
    def __init__(self, spec: SetupSpec, handle, info, device, coords, bnd):
        self.spec = spec
        self.h = handle
        self.info = info
        self.bytes = info["device_bytes"]
        self.coords = coords       # (M, dim) kept points on the device
        self.bnd = bnd             # (Mb, 2) boundary points or None
        self.last_use = time.perf_counter()
        self.inflight = 0
        self.graphs = {}           # bucket -> (graph, b_buf, x_buf)


class Server:
    def __init__(self, budget_bytes: int, nslots: int = 4, use_graphs: bool = True, device=None,
                 keep_results: bool = False, precision: int = AZ_MIXED, warm_process: bool = True):
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.setup_stream = torch.cuda.Stream(device=self.dev)
        self.keep_results = keep_results
        self.results = {}                  # rid -> (nrhs, N) solution columns (keep_results)
        self.budget = int(budget_bytes)
        self.used = 0
        self.setups: dict = {}
        self.queue: collections.OrderedDict = collections.OrderedDict()   # key -> deque of requests
        self.slots = [torch.cuda.Stream(device=self.dev) for _ in range(nslots)]
        self.slot_busy = [None] * nslots   # (event, setup, requests, x_buf, ncols) or None
        self.use_graphs = use_graphs
        self.rejections = 0
        self.setup_builds = 0
        self.evictions = 0
        self.high_water = 0
        self.precision = precision
        self.build_ms = []                 # wall time of each setup build (host view)
        self.pending_capture = collections.deque()   # (setup key, bucket) solved eagerly, not yet captured
        # process warm-up: library handles and kernels of the right-hand-side
        # generator, and one tiny setup and solve of each kind (first launches
        # load kernels), so that the first request does not pay for them
        a = torch.ones((8, 2), dtype=torch.float64, device=self.dev)
        torch.cos(a @ a.T).sum().item()
        if warm_process:
            self._warm_process()

    # ------------------------------------------------------------------ setups
    def _warm_process(self):
        th = 2 * np.pi * np.arange(16) / 16
        tiny = [SetupSpec(("warm1d",), 1, (64,), (2,), (1.0,), "approx", lambda x: (x >= -0.5) & (x <= 0.5), k=4),
                SetupSpec(("warm2d",), 2, (16, 16), (2, 2), (1.0, 1.0), "approx", star_fn(0.5, 0.1, 5), k=4),
                SetupSpec(("warmp",), 2, (16, 16), (2, 2), (1.0, 1.0), "poisson", star_fn(0.5, 0.1, 5),
                          np.stack([0.5 * np.cos(th), 0.5 * np.sin(th)], 1), 10.0, k=4)]
        builds = len(self.build_ms)
        for spec in tiny:
            st = self._build(spec)
            if st is None:
                continue
            _, b_buf, x_buf = self._graph(st, BUCKETS[0], self.slots[0], capture=False)
            self._rhs(st, [Request(-1, 0.0, spec, 1, 0)], b_buf)
            self._solve_fn(st, b_buf, x_buf, self.slots[0])
            torch.cuda.synchronize(self.dev)
            self._evict(st)
        # the warm-up is not part of the served workload's statistics
        del self.build_ms[builds:]
        self.setup_builds = 0
        self.evictions = 0
        self.high_water = 0
        self.pending_capture.clear()

    def _grid_coords(self, spec):
        """Oversampled grid coordinates per dimension, on the device (FP64)."""
        cs = []
        for d in range(spec.dim):
            L = spec.n[d] * spec.s[d]
            cs.append(-spec.T[d] + torch.arange(L, dtype=torch.float64, device=self.dev) * (2 * spec.T[d] / L))
        return cs

    def _build(self, spec: SetupSpec):
        t_build = time.perf_counter()
        opts = make_options(self.precision, spec.k, 1e-8, 0.0, 1, 1 if self.precision == AZ_MIXED else 0)
        grid = make_grid(spec.dim, spec.n, spec.s, spec.T)
        # domain mask and kept points evaluated on the device
        cs = self._grid_coords(spec)
        if spec.dim == 1:
            sel = spec.mask_fn(cs[0])
            pts = cs[0][sel][:, None]
        else:
            X, Y = torch.meshgrid(cs[0], cs[1], indexing="ij")
            sel = spec.mask_fn(X, Y).reshape(-1)
            pts = torch.stack([X.reshape(-1)[sel], Y.reshape(-1)[sel]], 1)
        mt = sel.to(torch.uint8)
        M = int(pts.shape[0])
        nb = 0 if spec.boundary is None else len(spec.boundary)
        need = az_query_footprint(grid, M, nb, opts, 64)
        if need > self.budget:
            return None
        # evict least-recently-used idle setups until the new one fits
        while self.used + need > self.budget:
            idle = [s for s in self.setups.values() if s.inflight == 0]
            if not idle:
                return None
            victim = min(idle, key=lambda s: s.last_use)
            self._evict(victim)
        bnd = None
        kernel = AZ_GAUSS
        if spec.kind == "poisson":
            kernel = AZ_NEG_LAPLACE_GAUSS
            bnd = torch.from_numpy(np.ascontiguousarray(spec.boundary)).to(self.dev)
        self.setup_stream.wait_stream(torch.cuda.current_stream(self.dev))
        h = az_setup(grid, mt, spec.epsh / (2 * spec.T[0] / spec.n[0]), kernel, bnd, spec.weight, opts,
                     self.setup_stream)
        info = az_get_info(h)
        st = _Setup(spec, h, info, self.dev, pts.contiguous(), bnd)
        self.setups[spec.key] = st
        self.used += st.bytes
        self.setup_builds += 1
        self.high_water = max(self.high_water, self.used)
        self.build_ms.append(1000.0 * (time.perf_counter() - t_build))
        return st

    def warm(self, specs, buckets=BUCKETS):
        """Build the given setups and capture their solve graphs before serving."""
        t0 = time.perf_counter()
        for spec in specs:
            st = self.setups.get(spec.key) or self._build(spec)
            if st is None:
                continue
            for b in buckets:
                self._graph(st, b, self.slots[0])
        torch.cuda.synchronize(self.dev)
        return 1000.0 * (time.perf_counter() - t0)

    def _evict(self, st: _Setup):
        st.graphs.clear()
        az_destroy(st.h)
        self.used -= st.bytes
        del self.setups[st.spec.key]
        self.evictions += 1

    def close(self):
        torch.cuda.synchronize(self.dev)
        for st in list(self.setups.values()):
            self._evict(st)

    # ------------------------------------------------------------------ solves
    @staticmethod
    def _offsets(reqs):
        """First column of each request in a batch, and the batch width.  Every
        request starts on an even column: the solver packs two real columns into
        one complex transform, so a request's columns then pair with each other
        (and an odd last column with a zero column) exactly as when it runs
        alone, and its result does not depend on the rest of the batch."""
        offs, col = [], 0
        for r in reqs:
            offs.append(col)
            col += r.nrhs + (r.nrhs & 1)
        return offs, col

    def _rhs(self, st: _Setup, reqs, out):
        """Fill out with each request's right-hand sides (cos(w.x + phi)) at its
        column offset; returns the batch width."""
        offs, width = self._offsets(reqs)
        for r, col in zip(reqs, offs):
            g = np.random.default_rng(r.seed)
            w = torch.from_numpy(g.uniform(1.0, 20.0, (r.nrhs, st.spec.dim))).to(self.dev)
            ph = torch.from_numpy(g.uniform(0.0, 2 * math.pi, r.nrhs)).to(self.dev)
            vals = torch.cos(st.coords @ w.T + ph[None, :])            # (M, nrhs)
            if st.spec.kind == "poisson":
                # interior data f = -Lap u = |w|^2 cos, then the Dirichlet data
                # u on the boundary points; az_collocate applies the row scaling
                lap = (w * w).sum(1)
                bvals = torch.cos(st.bnd @ w.T + ph[None, :])
                vals = torch.cat([vals * lap[None, :], bvals], 0)
            out[col:col + r.nrhs, :vals.shape[0]] = vals.T
        return width

    def _solve_fn(self, st, b_buf, x_buf, stream):
        if st.spec.kind == "poisson":
            M = st.info["M"]
            az_collocate(st.h, b_buf[:, :M], b_buf[:, M:], x_buf, stream)
        else:
            az_solve(st.h, b_buf, x_buf, stream)

    def _graph(self, st: _Setup, bucket: int, stream, capture: bool = True):
        """(graph or None, b_buf, x_buf) of a bucket; captures only when asked."""
        ent = st.graphs.get(bucket)
        if ent is None:
            rows = st.info["M"] + st.info["Mb"]
            b_buf = torch.zeros((bucket, rows), dtype=torch.float64, device=self.dev)
            x_buf = torch.zeros((bucket, st.info["N"]), dtype=torch.float64, device=self.dev)
            ent = (None, b_buf, x_buf)
            st.graphs[bucket] = ent
            if self.use_graphs and not capture:
                self.pending_capture.append((st.spec.key, bucket))
        if ent[0] is None and self.use_graphs and capture:
            _, b_buf, x_buf = ent
            with torch.cuda.stream(stream):
                self._solve_fn(st, b_buf, x_buf, stream)           # warm up (attribute set-up)
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                self._solve_fn(st, b_buf, x_buf, torch.cuda.current_stream())
            ent = (graph, b_buf, x_buf)
            st.graphs[bucket] = ent
        return ent

    def _capture_one(self):
        """Capture one deferred graph (called only while the server is idle)."""
        while self.pending_capture:
            key, bucket = self.pending_capture.popleft()
            st = self.setups.get(key)
            if st is not None and bucket in st.graphs and st.graphs[bucket][0] is None:
                self._graph(st, bucket, self.slots[0], capture=True)
                return

    def _dispatch(self, slot: int, key, now_fn):
        q = self.queue[key]
        st = self.setups.get(key)
        if st is None:
            st = self._build(q[0].spec)
            if st is None:
                while q:
                    r = q.popleft()
                    r.rejected = True
                    r.t_done = now_fn()
                    self.rejections += 1
                del self.queue[key]
                return
        reqs, ncols = [], 0
        while q and ncols + q[0].nrhs + (q[0].nrhs & 1) <= BUCKETS[-1]:
            r = q.popleft()
            reqs.append(r)
            ncols += r.nrhs + (r.nrhs & 1)
        if not q:
            del self.queue[key]
        bucket = next(b for b in BUCKETS if b >= ncols)
        stream = self.slots[slot]
        graph, b_buf, x_buf = self._graph(st, bucket, stream, capture=False)
        with torch.cuda.stream(stream):
            b_buf.zero_()
            self._rhs(st, reqs, b_buf)
            if graph is not None:
                graph.replay()
            else:
                self._solve_fn(st, b_buf, x_buf, stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        st.inflight += 1
        st.last_use = time.perf_counter()
        self.slot_busy[slot] = (ev, st, reqs, x_buf, ncols)

    def _poll(self, now_fn):
        for i, busy in enumerate(self.slot_busy):
            if busy is not None and busy[0].query():
                ev, st, reqs, x_buf, ncols = busy
                t = now_fn()
                offs, _ = self._offsets(reqs)
                for r, col in zip(reqs, offs):
                    r.t_done = t
                    if self.keep_results:
                        self.results[r.rid] = x_buf[col:col + r.nrhs].clone()
                st.inflight -= 1
                self.slot_busy[i] = None

    def run(self, requests, realtime: bool = True):
        """Serve the requests (sorted by arrival).  Returns the summary dict."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        i = 0
        n = len(reqs)
        while True:
            t = now()
            while i < n and (reqs[i].arrival <= t or not realtime):
                r = reqs[i]
                self.queue.setdefault(r.spec.key, collections.deque()).append(r)
                i += 1
                if not realtime and len(self.queue) > 64:
                    break
            self._poll(now)
            for s in range(len(self.slots)):
                if self.slot_busy[s] is None and self.queue:
                    # oldest waiting setup first; a setup already running on
                    # another slot is skipped so its batch can keep growing
                    keys = [k for k in self.queue
                            if not any(b is not None and b[1].spec.key == k for b in self.slot_busy)]
                    if keys:
                        self._dispatch(s, keys[0], now)
            idle = all(b is None for b in self.slot_busy)
            if i >= n and not self.queue and idle:
                break
            if idle and not self.queue and self.pending_capture:
                self._capture_one()
                continue
            if realtime and i < n and not self.queue and idle:
                time.sleep(max(0.0, min(0.001, reqs[i].arrival - now())))
        elapsed = now()
        done = [r for r in reqs if not r.rejected]
        lat = sorted(1000.0 * (r.t_done - r.arrival) for r in done)
        solves = sum(r.nrhs for r in done)

        def pct(q):
            return lat[min(len(lat) - 1, int(q * len(lat)))] if lat else None
        return {"requests": n, "served": len(done), "rejected": self.rejections, "rhs_solved": solves,
                "elapsed_s": elapsed, "solves_per_s": solves / elapsed if elapsed > 0 else None,
                "latency_ms": {"p50": pct(0.50), "p99": pct(0.99), "max": lat[-1] if lat else None},
                "setup_builds": self.setup_builds, "evictions": self.evictions,
                "build_ms": {"p50": float(np.median(self.build_ms)) if self.build_ms else None,
                             "max": max(self.build_ms) if self.build_ms else None},
                "precision": "mixed" if self.precision == AZ_MIXED else "fp64",
                "device_bytes_high_water": self.high_water}


# --------------------------------------------------------------------------- the mixed workload
def star_fn(r0, a, k):
    """Star domain r(theta) = r0 + a cos(k theta) (numpy or torch coordinates)."""
    def f(X, Y):
        if isinstance(X, torch.Tensor):
            return torch.sqrt(X * X + Y * Y) <= r0 + a * torch.cos(k * torch.atan2(Y, X))
        return np.sqrt(X * X + Y * Y) <= r0 + a * np.cos(k * np.arctan2(Y, X))
    return f


def setup_pool(seed: int, count: int = 32, max2d: int = 512):
    """A seeded pool of setups with the stream's mix of problem kinds."""
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(count):
        u = rng.random()
        if u < 0.4:
            N = 1 << int(rng.integers(12, 19))
            a = float(rng.uniform(-1.0, 0.0))
            spec = SetupSpec(("1d", N, round(a, 6)), 1, (N,), (2,), (1.0,), "approx",
                             (lambda a: (lambda x: (x >= a) & (x <= a + 1.0)))(a), k=24)
        elif u < 0.8:
            n = int(rng.choice([64, 128, 256, 512]))
            n = min(n, max2d)
            a, kk = float(rng.uniform(0.0, 0.2)), int(rng.integers(3, 8))
            spec = SetupSpec(("2d", n, round(a, 6), kk), 2, (n, n), (2, 2), (1.0, 1.0), "approx",
                             star_fn(0.5, a, kk), k=64)
        else:
            n = int(rng.choice([64, 128, 256]))
            a, kk = float(rng.uniform(0.0, 0.2)), int(rng.integers(3, 8))
            th = 2 * np.pi * np.arange(512) / 512
            r = 0.5 + a * np.cos(kk * th)
            spec = SetupSpec(("poisson", n, round(a, 6), kk), 2, (n, n), (2, 2), (1.0, 1.0), "poisson",
                             star_fn(0.5, a, kk), np.stack([r * np.cos(th), r * np.sin(th)], 1), 10.0, k=64)
        pool.append(spec)
    return pool


def poisson_stream(seed: int, rate: float, duration: float, pool):
    """Poisson arrivals at `rate` per second for `duration` seconds, 1..32 RHS each."""
    rng = np.random.default_rng(seed + 1)
    t, rid, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        spec = pool[int(rng.integers(0, len(pool)))]
        out.append(Request(rid, t, spec, int(rng.integers(1, 33)), int(rng.integers(0, 2 ** 31))))
        rid += 1
    return out
