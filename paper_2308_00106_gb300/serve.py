"""Continuous-batching serving loop over resident permuted matrices.

The paper motivates permutation as a one-time cost amortised over reuse of a
matrix (Section 1, the preconditioning analogy); serving keeps many permuted
matrices resident on the GPU and answers a stream of requests against them:

  spmv   y' = A' x'             (one product)
  spmm   Y' = A' X', k = 2..32  (one product)
  power  20 steps of u <- Q(A' u) / ||A' u||, then lambda = u . Q(A' u)
         (Q = P_c^{-1} P_r^{-1}: the power iteration of A, kept in the permuted
         space; not in the paper)

Vectors are in the permuted space (clients reuse the matrix iteratively).  The
scheduler runs on the host and only decides what to launch; every product runs
in the library's batched persistent kernel (maxe_batch_run) and every vector
step in its kernels (maxe_vec_norm_gather / maxe_vec_dot_gather).

Continuous batching: requests are admitted as soon as their buffers fit under
the device-memory cap (and while the admitted work waiting for a step is under
about two steps per stream, so admitting interleaves with launching); each
batch step takes one unit of work (a product) from
admitted requests that are not already on the GPU, oldest first, up to a byte
budget of work per step, so requests join and leave between steps and a power
iteration advances one product per step.  Two CUDA streams, each with its own
batch object, keep two steps in flight, so a step's work overlaps the previous
one on the device.  Every matrix has a fixed
batch plan, so a request's result is bit-identical alone and in any mix.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import maxe


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the trace starts
    mat: int
    kind: str  # "spmv" | "spmm" | "power"
    k: int = 1
    steps: int = 20
    seed: int = 0
    # filled in by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    units_done: int = 0
    result: object = None
    bufs: dict = field(default_factory=dict)

    @property
    def units(self) -> int:
        return self.steps + 1 if self.kind == "power" else 1

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def make_trace(n: int, n_mats: int, rate: float, seed: int = 0, mix=(0.6, 0.3, 0.1), kmax: int = 32,
               steps: int = 20):
    """Poisson arrivals (rate requests/s; rate = inf puts all at t = 0), uniform matrix choice,
    request kinds by `mix` (spmv, spmm, power), SpMM k ~ U{2..kmax}."""
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / rate, n) if math.isfinite(rate) else np.zeros(n)
    t = np.cumsum(gaps)
    kinds = g.choice(["spmv", "spmm", "power"], size=n, p=list(mix))
    reqs = []
    for i in range(n):
        kind = str(kinds[i])
        k = int(g.integers(2, kmax + 1)) if kind == "spmm" else 1
        reqs.append(Request(i, float(t[i]) if math.isfinite(rate) else 0.0, int(g.integers(0, n_mats)), kind, k,
                            steps if kind == "power" else 0, seed * 1_000_003 + i))
    return reqs


def clone_request(r: Request, arrival: float = 0.0) -> Request:
    return Request(r.rid, arrival, r.mat, r.kind, r.k, r.steps, r.seed)


class Server:
    """Resident permuted matrices + the continuous-batching loop."""

    def __init__(self, mats, seed: int = 2308, mem_cap_bytes: int = 60 << 30, streams: int = 2,
                 tune: bool = False, batch_capacity: int = 4096, step_bytes: int = 2 << 30,
                 autotune: bool = True, xslice: bool = False):
        maxe.load(build_if_missing=True)
        self.mats = mats
        self.handles, self.Q, self.perm_c = [], [], []
        resident = 0
        for m, A in enumerate(mats):
            r = maxe.maxe_build_permutation(seed + m, A.rows, 0)
            c = maxe.maxe_build_permutation(seed + m, A.cols, 1)
            # autotuned handles: the x-sliced SpMV where it is faster, and the
            # fastest SpMM kernel (which the handle's batch plan then takes);
            # xslice: the x-sliced form on every handle
            h = maxe.from_csr(A, r, c, autotune=autotune and not xslice, xslice=xslice)
            if tune:
                maxe.maxe_batch_tune(h, 1)
            self.handles.append(h)
            self.perm_c.append(c)
            if A.rows == A.cols:
                rinv = maxe.maxe_invert_permutation(r)
                self.Q.append(maxe.maxe_permute_gather(c, rinv))  # Q[j] = rinv[cperm[j]]
            else:
                self.Q.append(None)
            resident += A.nnz * (4 + A.val.element_size()) + (A.rows + 1) * 4 + (A.rows + A.cols) * 4 * 2
        torch.cuda.synchronize()
        self.resident_bytes = resident
        self.mem_cap = mem_cap_bytes
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.adm_stream = torch.cuda.Stream()  # initialises admitted requests' buffers
        self.batches = [maxe.Batch(batch_capacity, stream=s) for s in self.streams]
        self.capacity = batch_capacity
        self.step_bytes = step_bytes  # work per batch step, so that the streams alternate and overlap
        # admitted work waiting for a step is kept to about two steps per stream, so
        # that admitting (host allocations, input initialisation) interleaves with
        # launching instead of preceding it
        self.backlog_bytes = 2 * streams * step_bytes
        self.gen = torch.Generator(device="cuda")  # re-seeded per request

    # ---------------------------------------------------------------- helpers
    def request_bytes(self, r: Request) -> int:
        A = self.mats[r.mat]
        b = (A.cols + A.rows) * (1 if r.k == 1 else (r.k + 3) // 4 * 4) * 4
        if r.kind == "power":
            b += (A.cols + A.rows) * 4 + 1024 * 8
        return b

    def unit_bytes(self, r: Request) -> int:
        """Algorithmic bytes of one product of the request (every byte once)."""
        A = self.mats[r.mat]
        return A.nnz * (A.val.element_size() + 4) + (A.rows + 1) * 4 + (A.rows + A.cols) * r.k * 4

    def _admit(self, r: Request, stream):
        A = self.mats[r.mat]
        with torch.cuda.stream(stream):
            g = self.gen
            g.manual_seed(r.seed)
            if r.kind == "power":
                u = torch.rand(A.cols, generator=g, device="cuda") * 2 - 1
                r.bufs = {"u": u, "w": torch.empty(A.rows, device="cuda"),
                          "scratch": torch.empty(1024, dtype=torch.float64, device="cuda"),
                          "lam": torch.empty(1, dtype=torch.float64, device="cuda"), "u0": u.clone()}
            else:
                # 16-byte rows for k > 1 (the kernel gathers 4 columns per load); unit
                # strides for k = 1, which the batched kernel runs in its SpMV class
                kp = 1 if r.k == 1 else (r.k + 3) // 4 * 4
                if kp == r.k:
                    X = torch.rand(A.cols, r.k, generator=g, device="cuda").mul_(2).sub_(1)
                else:
                    X = torch.zeros(A.cols, kp, device="cuda")
                    X[:, :r.k] = torch.rand(A.cols, r.k, generator=g, device="cuda") * 2 - 1
                r.bufs = {"X": X[:, :r.k], "Y": torch.empty(A.rows, kp, device="cuda")[:, :r.k]}

    def _launch(self, si: int, reqs):
        """One step on stream si: the products of `reqs` (single SpMV launches
        where the handle runs the x-sliced form, which one persistent batched
        launch would not use; one batched launch per kernel class for the
        rest), then the power iterations' vector steps."""
        s = self.streams[si]
        items, singles = [], []
        for r in reqs:
            h = self.handles[r.mat]
            if r.kind == "power":
                x, y = r.bufs["u"], r.bufs["w"]
            else:
                x, y = r.bufs["X"], r.bufs["Y"]
            if (r.kind == "power" or r.k == 1) and h.xslice():
                singles.append((h, x.reshape(-1), y.reshape(-1)))
            else:
                items.append((h, x, y, False))
        b = self.batches[si]
        b.set(items)
        b.run(stream=s)
        for h, x, y in singles:
            maxe.maxe_spmv(h, x, y, permuted=True, stream=s)
        with torch.cuda.stream(s):
            for r in reqs:
                if r.kind != "power":
                    continue
                if r.units_done < r.steps:  # normalise: u <- Q(w) / ||w||
                    maxe.maxe_vec_norm_gather(self.Q[r.mat], r.bufs["w"], r.bufs["u"], r.bufs["scratch"], stream=s)
                else:  # lambda = u . Q(w)
                    maxe.maxe_vec_dot_gather(self.Q[r.mat], r.bufs["u"], r.bufs["w"], r.bufs["scratch"],
                                             r.bufs["lam"], stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return ev

    def _finish(self, r: Request, keep: bool):
        if keep:
            if r.kind == "power":
                r.result = (float(r.bufs["lam"].item()), r.bufs["u"].clone(), r.bufs["u0"])
            else:
                r.result = r.bufs["Y"].contiguous()
            # The copies above are queued on the current stream, but the buffers
            # belong to adm_stream: once dropped, the caching allocator may hand
            # them to the next admission on adm_stream, so that stream must not
            # run ahead of the copies.
            self.adm_stream.wait_stream(torch.cuda.current_stream())
        r.bufs = {}

    # ------------------------------------------------------------ the loop
    def run(self, trace, keep_results: bool = False, max_wall: float = 600.0, max_items: int | None = None):
        """Serve `trace` (requests sorted by arrival); returns a stats dict.
        max_items caps the requests per batch step (1 = no batching)."""
        cap_items = self.capacity if max_items is None else max(1, min(max_items, self.capacity))
        trace = sorted(trace, key=lambda r: r.arrival)
        n = len(trace)
        for r in trace:
            if self.request_bytes(r) > self.mem_cap - self.resident_bytes:
                raise ValueError(f"request {r.rid} needs more device memory than the cap leaves")
        waiting = collections.deque()
        ready = collections.deque()
        inflight = {}  # stream index -> (event, requests)
        mem_used = 0
        ready_work = 0  # unit bytes of admitted requests waiting for a step
        nxt = done = 0
        bytes_done = 0
        steps = 0
        peak_mem = 0
        max_batch = 0
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            if now > max_wall:
                raise TimeoutError("serving trace did not finish")
            progressed = False
            while nxt < n and trace[nxt].arrival <= now:
                waiting.append(trace[nxt])
                nxt += 1
            while (waiting and mem_used + self.request_bytes(waiting[0]) <= self.mem_cap - self.resident_bytes
                   and ready_work < self.backlog_bytes):
                r = waiting.popleft()
                mem_used += self.request_bytes(r)
                peak_mem = max(peak_mem, mem_used)
                self._admit(r, self.adm_stream)
                r.t_admit = time.perf_counter() - t0
                ready.append(r)
                ready_work += self.unit_bytes(r)
                progressed = True
            for si in list(inflight):
                ev, reqs = inflight[si]
                if not ev.query():
                    continue
                del inflight[si]
                tnow = time.perf_counter() - t0
                for r in reqs:
                    r.units_done += 1
                    bytes_done += self.unit_bytes(r)
                    if r.units_done >= r.units:
                        r.t_done = tnow
                        self._finish(r, keep_results)
                        mem_used -= self.request_bytes(r)
                        done += 1
                    else:
                        ready.append(r)
                        ready_work += self.unit_bytes(r)
                progressed = True
            for si in range(len(self.streams)):
                if si in inflight or not ready:
                    continue
                take, work = [], 0
                while ready and len(take) < cap_items and (not take or work < self.step_bytes):
                    r = ready.popleft()
                    take.append(r)
                    work += self.unit_bytes(r)
                ready_work -= work
                # the first step of a freshly admitted request must see its initialised buffers
                self.streams[si].wait_stream(self.adm_stream)
                inflight[si] = (self._launch(si, take), take)
                steps += 1
                max_batch = max(max_batch, len(take))
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in trace])
        by = {}
        for kind in ("spmv", "spmm", "power"):
            v = np.array([r.latency for r in trace if r.kind == kind])
            if v.size:
                by[kind] = {"n": int(v.size), "p50_ms": float(np.percentile(v, 50) * 1e3),
                            "p99_ms": float(np.percentile(v, 99) * 1e3)}
        return {"requests": n, "wall_s": wall, "req_per_s": n / wall, "gbs": bytes_done / wall / 1e9,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "by_kind": by, "batch_steps": steps, "max_batch": max_batch, "peak_request_bytes": peak_mem,
                "resident_bytes": self.resident_bytes}

    def close(self):
        for b in self.batches:
            b.close()
        for h in self.handles:
            h.close()
