#!/usr/bin/env python
"""SpMV GB/s and fraction of the HBM roofline on the 1M-row power-law matrix,
permuted (rows and columns randomly permuted, arXiv 2308.00106 Eq. 1) vs plain.

One step = one product y' = A' x' on the resident permuted matrix with the
vectors kept in the permuted space (the iterative reuse the paper targets).
The permutation preprocessing (keys, sort, permute_csr, entropy) runs once
before the timed region and is reported separately.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl maxe|reference]
                    [--workload powerlaw|laplacian|blockdiag]

Multi-GPU (torchrun, one rank per GPU): the path does not shard, each rank runs
an independent replica ("replicas only"), value = bytes of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s & frac of HBM roofline, permuted vs plain; served p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def alg_bytes(M, N, Z, vbytes, xbytes, ybytes, k=1):
    """Algorithmic bytes of one CSR product: every byte counted once."""
    return Z * (vbytes + 4) + (M + 1) * 4 + M * k * ybytes + N * k * xbytes


# The ncu DRAM traffic quoted in the roofline belongs to one revision of a
# kernel's source: each record under profiles/ carries the SHA-256 of the
# source files it was measured on, and a record whose hash differs from the
# current files is not quoted (traffic null).
KERNEL_SOURCES = {
    "spmv_xslice_kernel": ["paper_2308_00106_gb300/csrc/xslice.cu", "paper_2308_00106_gb300/csrc/internal.cuh"],
    "spmm_warp_kernel": ["paper_2308_00106_gb300/csrc/spmv_warp.cuh", "paper_2308_00106_gb300/csrc/spmv.cu",
                         "paper_2308_00106_gb300/csrc/internal.cuh"],
}
PROFILE_RECORD = {"spmv_xslice_kernel": "spmv_xslice_powerlaw1M_f32.json",
                  "spmm_warp_kernel": "spmv_warp_powerlaw1M_f32.json"}


def kernel_source_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_from_record(kernel: str, profiles_dir=None):
    """DRAM bytes per launch of `kernel` from its committed ncu record, or None
    when there is none or it was measured on other sources."""
    p = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), PROFILE_RECORD[kernel])
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    if rec.get("source_sha256") != kernel_source_hash(kernel):
        return None
    return float(rec["traffic_bytes_per_launch"])


def record_profile(csv_path: str, kernel: str, launch: int, command: str, workload: str, out_dir=None) -> dict:
    """Write the ncu record of `kernel` (DRAM read + write bytes of its
    `launch`-th captured launch, from `ncu -i REP --page raw --csv` output) with
    the hash of the current sources."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    head = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "dram__bytes_read.sum" in r)
    cols, units = rows[head], rows[head + 1]
    data = [r for r in rows[head + 2:] if len(r) == len(cols) and kernel in r[cols.index("Kernel Name")]]
    r = data[launch]
    scale = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "nsecond": 1, "usecond": 1e3, "msecond": 1e6,
             "ns": 1, "us": 1e3, "ms": 1e6}

    def val(name):
        i = cols.index(name)
        return float(r[i].replace(",", "")) * scale[units[i].strip().lower()]

    rec = {"kernel": kernel, "kernel_name": r[cols.index("Kernel Name")], "workload": workload,
           "traffic_bytes_per_launch": val("dram__bytes_read.sum") + val("dram__bytes_write.sum"),
           "dram_read_bytes": val("dram__bytes_read.sum"), "dram_write_bytes": val("dram__bytes_write.sum"),
           "duration_us_under_ncu": val("gpu__time_duration.sum") / 1e3 if "gpu__time_duration.sum" in cols else None,
           "note": "ncu times are serialised and cold-cache; the bench's CUDA-event timing is the performance number",
           "source_files": KERNEL_SOURCES[kernel], "source_sha256": kernel_source_hash(kernel), "command": command}
    with open(os.path.join(out_dir or os.path.join(ROOT, "profiles"), PROFILE_RECORD[kernel]), "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    return rec


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.file.name)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] >= 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2][1:5]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    """The largest of the ranks' values (timings: the slowest replica sets the job's time)."""
    if world == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput of independent replicas: the units all ranks processed
    divided by the slowest rank's time (units per second)."""
    return units_per_rank * world / (ms_max * 1e-3)


def make_workload(name, seed, device):
    from paper_2308_00106_gb300 import workloads as W
    if name == "powerlaw":
        return W.powerlaw(seed, device=device), "f32", (
            "power-law CSR 1048576x1048576, row lengths Zipf(1.5) on 1..1000, columns i+round(N(0,2000)), "
            "FP32 values U[-1,1], int32 indices")
    if name == "laplacian":
        return W.laplacian5(4096, "f32", device), "f32", "5-point Laplacian on a 4096x4096 grid, FP32, natural order"
    if name == "blockdiag":
        return W.blockdiag(seed, device=device), "f64", (
            "4096x4096, 16 diagonal 256x256 blocks at 2% fill + 2000 off-block entries, FP64")
    if name == "clustered":
        return W.clustered_heavy(seed, 1 << 20, dtype="f32", device=device), "f32", (
            "1048576x1048576, first 1% of rows 1000 entries, the rest 16, distinct uniform columns, FP32")
    raise SystemExit(f"unknown workload {name}")


def timed_steps(step, K, W, world, graph_len=50):
    """W warm-up steps, then exactly K steps (CUDA graph replays of graph_len
    steps plus a remainder, when K >= graph_len > 1; else K eager launches)
    bracketed by barrier + synchronize; returns (ms per step, graph replayed)."""
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    g = None
    graph_len = min(graph_len, K)
    if graph_len > 1:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()  # warm the capture stream
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(graph_len):
                step()
        g.replay()
        torch.cuda.synchronize()
    reps, rem = (K // graph_len, K % graph_len) if g is not None else (0, K)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    for _ in range(rem):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    return max_over_ranks(ms, world) / K, g is not None


def seed_sweep(A, x, args, world, tune):
    """The paper's protocol (32 runs with different permutations): permuted SpMV
    for seeds 0..n-1, each with its own handle (built as in the timed run),
    GB/s min / mean / max, the 64x64-grid entropy per seed, and the cold first
    launch of the first seed (right after its handle is built, L2 flushed)."""
    from paper_2308_00106_gb300 import maxe
    M, N = A.rows, A.cols
    vb = {torch.float64: 8, torch.float32: 4, torch.bfloat16: 2}[A.val.dtype]
    xb = 8 if vb == 8 else 4
    by = alg_bytes(M, N, A.nnz, vb, xb, xb)
    gbs, ents, cold = [], [], None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for sd in range(args.seeds):
        r = maxe.maxe_build_permutation(sd, M, 0)
        c = maxe.maxe_build_permutation(sd, N, 1)
        h = maxe.from_csr(A, r, c, autotune=tune)
        xp = x[c.long()].contiguous()
        y = torch.empty(M, dtype=xp.dtype, device="cuda")
        if sd == 0:
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            maxe.maxe_spmv(h, xp, y, permuted=True)
            e1.record()
            torch.cuda.synchronize()
            cold = e0.elapsed_time(e1)
        ms, _ = timed_steps(lambda: maxe.maxe_spmv(h, xp, y, permuted=True), 200, 3, world, graph_len=50)
        gbs.append(by / (ms * 1e-3) / 1e9)
        ents.append(maxe.maxe_nnz_entropy(h, 64, 64, counts=False)[0])
        h.close()
    del flush
    return {"n": args.seeds, "gbs_min": round(min(gbs), 3), "gbs_mean": round(float(np.mean(gbs)), 3),
            "gbs_max": round(max(gbs), 3), "entropy_64x64_min": round(min(ents), 4),
            "entropy_64x64_max": round(max(ents), 4), "cold_first_launch_ms": cold,
            "what": "seeds 0..n-1 for the row and column permutations; 200 products each (CUDA graph)"}


def timed_streams(step, streams, K, W, world, host_ms=None):
    """W warm-up steps, then exactly K steps step(k) that spread over `streams`;
    device time from an event before the first to one after all streams drain
    (barrier + synchronize on both sides); ms per step, max over ranks.  With a
    list host_ms, appends the host's time per step to enqueue the K steps."""
    for k in range(W):
        step(k)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for st in streams:
        st.wait_event(e0)
    t0 = time.perf_counter()
    for k in range(K):
        step(k)
    if host_ms is not None:
        host_ms.append((time.perf_counter() - t0) * 1e3 / K)
    for st in streams:
        cur.wait_stream(st)
    e1.record(cur)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1), world) / K


def flushed_launch_ms(step, reps=20):
    """Median device time of one launch with L2 flushed (256 MB write) before each."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    times = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    del flush
    return statistics.median(times)


def host_info() -> dict:
    """CPU model and core count of the machine the CPU numbers come from."""
    import platform
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def cpu_baseline(A, x_np, code, seconds=10.0):
    """The oracle's FP64 CSR product on the host (one core), bounded to ~`seconds`;
    returns (seconds per product, products timed, the oracle's y)."""
    import oracle
    rp, co, va = A
    t0 = time.perf_counter()
    y = oracle.spmv(len(rp) - 1, rp, co, va, code, x_np)
    t1 = time.perf_counter() - t0
    reps = max(1, int(seconds / max(t1, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.spmv(len(rp) - 1, rp, co, va, code, x_np)
    return (time.perf_counter() - t0) / reps, reps, y


def run_reference(args):
    """Reference arm: the CPU oracle timed as it stands on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2308_00106_gb300 import workloads as W
    oracle.build()
    # the same matrix as the GPU arm: generated by the same torch stream (on the
    # GPU when there is one; input generation only, outside the timed region)
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, dtype, desc = make_workload(args.workload, args.seed, gen_dev)
    A = A.to("cpu")
    rp, co, va = A.numpy()
    M, N, Z = A.rows, A.cols, A.nnz
    rperm = oracle.build_permutation(args.seed, M, 0)
    cperm = oracle.build_permutation(args.seed, N, 1)
    prp, pco, pva = oracle.permute_csr(M, N, rp, co, va, W.DTYPE_CODE[dtype], rperm, cperm)
    x = W.vector(1, N, "f64", "cpu").numpy()
    code = W.DTYPE_CODE[dtype]
    t0 = time.perf_counter()
    oracle.spmv(M, prp, pco, pva, code, x)
    t_full = time.perf_counter() - t0
    budget = 150.0  # seconds for the whole run
    frac = min(1.0, budget / max(1, args.steps + args.warmup) / max(t_full, 1e-6))
    r1 = max(1, int(M * frac))
    sub = (prp[:r1 + 1], pco[:prp[r1]], pva[:prp[r1]])
    for _ in range(args.warmup):
        oracle.spmv(r1, *sub, code, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(r1, *sub, code, x)
    dt = (time.perf_counter() - t0) / args.steps
    vb = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
    xb = 8 if dtype == "f64" else 4
    z1 = int(prp[r1])
    cores = 1
    pool = None
    if args.cpu_workers > 1:
        # the paper's parallel CPU CSR (Section 6): rows split into equal-row
        # ranges, one per worker; here threads (the oracle's C call releases the
        # GIL), the same sample of rows, natural order and permuted order
        import concurrent.futures as cf
        nw = args.cpu_workers

        def ranges(rp_, co_, va_):
            cuts = [r1 * w // nw for w in range(nw + 1)]
            out = []
            for a, b in zip(cuts[:-1], cuts[1:]):
                e0, e1 = int(rp_[a]), int(rp_[b])
                out.append((b - a, (rp_[a:b + 1] - e0).astype(np.int32), co_[e0:e1], va_[e0:e1]))
            return out

        def timed_pool(parts):
            with cf.ThreadPoolExecutor(nw) as ex:
                run = lambda: list(ex.map(lambda q: oracle.spmv(q[0], q[1], q[2], q[3], code, x), parts))  # noqa: E731
                for _ in range(args.warmup):
                    run()
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    run()
                return (time.perf_counter() - t0) / args.steps

        dt_perm = timed_pool(ranges(prp, pco, pva))
        dt_nat = timed_pool(ranges(rp, co, va))
        z_nat = int(rp[r1])
        pool = {"workers": nw, "split": "equal rows", "permuted_ms": dt_perm * 1e3, "natural_ms": dt_nat * 1e3,
                "natural_gbs": round(alg_bytes(r1, N, z_nat, vb, xb, xb) / dt_nat / 1e9, 4),
                "permuted_over_natural_speed": round(dt_nat / dt_perm * (z1 / max(z_nat, 1)), 4)}
        dt = dt_perm
        cores = nw
    gbs = alg_bytes(r1, N, z1, vb, xb, xb) / dt / 1e9
    sample = f"rows 0..{r1} of the permuted matrix ({z1} of {Z} nonzeros) per step"
    if pool:
        sample += f", split into {pool['workers']} equal-row ranges on as many threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "variant": "permuted R-C, vectors in permuted space", "nnz": Z,
                   "inputs": f"generated with torch on {gen_dev} (the GPU arm's stream when on cuda)"},
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        **({"equal_rows_pool": pool} if pool else {}),
    }))


def batched_measure(seed, count, steps, warmup, world, tune, profile=False):
    """256 uneven matrices with 1..16 right-hand sides: one persistent launch
    (CUDA graph) against per-matrix launches of the same kernel family.  Returns
    the measurement as a dict (None when profiling)."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    t0 = time.perf_counter()
    mats, ks = W.batched_set(seed, count=count, device="cuda")
    t_gen = time.perf_counter() - t0
    hs, Xs, Ys, Yp = [], [], [], []
    t0 = time.perf_counter()
    for m, (A, k) in enumerate(zip(mats, ks)):
        r = maxe.maxe_build_permutation(seed + m, A.rows, 0)
        c = maxe.maxe_build_permutation(seed + m, A.cols, 1)
        # the per-matrix launches and the default batch plan take the same SpMM
        # kernel (one row per lane group)
        h = maxe.from_csr(A, r, c, spmm_rows=True)
        if tune:
            maxe.maxe_batch_tune(h, k)
        hs.append(h)
        kp = 1 if k == 1 else (k + 3) // 4 * 4  # 16-byte rows for k > 1; unit strides for SpMV
        Xb = torch.zeros(A.cols, kp, device="cuda")
        Xb[:, :k] = W.matrix_rhs(m, A.cols, k, "f32", "cuda")
        Xs.append(Xb[:, :k])
        Ys.append(torch.empty(A.rows, kp, device="cuda")[:, :k])
        Yp.append(torch.empty(A.rows, kp, device="cuda")[:, :k])
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    total = sum(alg_bytes(A.rows, A.cols, A.nnz, 4, 4, 4, k) for A, k in zip(mats, ks))
    b = maxe.Batch(len(mats))
    b.set([(h, X, Y, False) for h, X, Y in zip(hs, Xs, Ys)])

    def step_batched():
        b.run()

    def step_permatrix():
        for h, X, Y in zip(hs, Xs, Yp):
            maxe.maxe_spmm(h, X, Y, permuted=True)

    if profile:
        for _ in range(3):
            step_batched()
        torch.cuda.synchronize()
        return None
    K = max(1, steps)
    ms_b, g_b = timed_steps(step_batched, K * 10, warmup, world, graph_len=10)
    ms_pm_graph, _ = timed_steps(step_permatrix, K, warmup, world, graph_len=1 if K < 2 else 2)
    ms_pm, _ = timed_steps(step_permatrix, K, warmup, world, graph_len=1)
    plans = [maxe.maxe_batch_plan_info(h) for h in hs]
    kernels = ["spmv16" if k == 1 and p[2] == 16 else "spmv8" if k == 1 else h.batch_spmm_kernel()
               for h, k, p in zip(hs, ks, plans)]
    # one persistent launch per kernel class present (the SpMM passes and lanes kernels share one)
    launches = len({"spmm" if kn in ("passes", "lanes") else kn for kn in kernels})
    hbm, src = peaks()
    gbs = total / (ms_b * 1e-3) / 1e9
    b.close()
    for h in hs:
        h.close()
    return {
        "value": round(gbs * world, 3), "unit": "GB/s", "ms_per_batch": ms_b,
        "config": {"workload": "256 square matrices, rows log-uniform 1k-200k, Poisson(U[8,64]) row lengths, "
                               "uniform distinct columns, FP32, k ~ U{1..16}, R-C permuted, vectors permuted",
                   "matrices": len(mats), "total_nnz": int(sum(A.nnz for A in mats)),
                   "rows_total": int(sum(A.rows for A in mats)), "alg_bytes_per_batch": total,
                   "timing": f"{K * 10} batches{' (CUDA graph of 10)' if g_b else ''}; per-matrix: {K} batches"},
        "per_matrix_launches": {"ms_per_batch_stream": ms_pm, "ms_per_batch_graph": ms_pm_graph,
                                "gbs_stream": round(total / (ms_pm * 1e-3) / 1e9, 3),
                                "gbs_graph": round(total / (ms_pm_graph * 1e-3) / 1e9, 3)},
        "over_per_matrix": round(ms_pm_graph / ms_b, 3),
        "over_per_matrix_stream": round(ms_pm / ms_b, 3),
        "roofline": {"bound": "hbm", "achieved": round(gbs, 3), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 4), "peak_source": src},
        "plans": {"entries_per_task": sorted({p[0] for p in plans})[:8],
                  "items16": sum(1 for p in plans if p[2] == 16), "tuned": bool(tune),
                  "kernels": {kn: kernels.count(kn) for kn in sorted(set(kernels))}},
        "gen_s": t_gen, "prep_and_tune_s": t_prep, "gpu_launches_per_batch": launches,
    }


def run_batched(args):
    from paper_2308_00106_gb300 import maxe

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    clocks = Clocks(local)
    clocks.start()
    out = batched_measure(args.seed, args.batch_count, max(1, args.steps // 100), args.warmup, world,
                          tune=not (args.profile or args.no_tune), profile=args.profile)
    clk = clocks.stop()
    if out is None:
        print(json.dumps({"profile": "done"}))
        return
    out = {"metric": "batched SpMV/SpMM GB/s (config: 256 uneven matrices, 1-16 RHS), one persistent launch vs "
                     "per-matrix launches", "n_gpus": world, "higher_is_better": True, "dtype": "f32",
           "data": "synthetic", **out, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def serving_measure(seed, requests, loads=(0.5, 0.8, 0.95), unbatched=True):
    """64 resident permuted matrices, Poisson request stream (60% SpMV, 30% SpMM
    k = 2..32, 10% 20-step power iteration), 60 GB device-memory cap: saturation
    throughput, p50/p99 latency at fractions of it, the same server without
    batching, and the same requests launched back to back with no scheduler."""
    from paper_2308_00106_gb300 import maxe, serve
    from paper_2308_00106_gb300 import workloads as W

    t0 = time.perf_counter()
    mats = W.serving_set(seed, device="cuda")
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    srv = serve.Server(mats, seed=seed, mem_cap_bytes=60 << 30)
    t_load = time.perf_counter() - t0
    n = requests
    # warm-up, then saturation: every request queued at t = 0
    srv.run(serve.make_trace(min(200, n), len(mats), math.inf, seed=1))
    sat = srv.run(serve.make_trace(n, len(mats), math.inf, seed=2))
    at = {}
    for f in loads:
        at[str(f)] = srv.run(serve.make_trace(n, len(mats), f * sat["req_per_s"], seed=3 + int(f * 100)))
    unb = None
    if unbatched:
        unb_sat = srv.run(serve.make_trace(n, len(mats), math.inf, seed=2), max_items=1)
        unb_loads = {}
        for f in loads[:2]:
            unb_loads[str(f)] = srv.run(serve.make_trace(n, len(mats), f * sat["req_per_s"], seed=3 + int(f * 100)),
                                        max_items=1)
        unb = {"saturation": {k: unb_sat[k] for k in ("req_per_s", "gbs", "p50_ms", "p99_ms")},
               "loads": {f: {k: v[k] for k in ("req_per_s", "gbs", "p50_ms", "p99_ms")} for f, v in unb_loads.items()},
               "throughput_over": round(sat["req_per_s"] / unb_sat["req_per_s"], 3)}
    # the same saturation trace served one request at a time with single-matrix launches
    trace = serve.make_trace(n, len(mats), math.inf, seed=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bytes_seq = 0
    scratch = torch.empty(1024, dtype=torch.float64, device="cuda")
    lam = torch.empty(1, dtype=torch.float64, device="cuda")
    for r in trace:
        A, h = mats[r.mat], srv.handles[r.mat]
        if r.kind == "power":
            u = torch.rand(A.cols, device="cuda") * 2 - 1
            w = torch.empty(A.rows, device="cuda")
            for _ in range(r.steps):
                maxe.maxe_spmv(h, u, w, permuted=True)
                maxe.maxe_vec_norm_gather(srv.Q[r.mat], w, u, scratch)
            maxe.maxe_spmv(h, u, w, permuted=True)
            maxe.maxe_vec_dot_gather(srv.Q[r.mat], u, w, scratch, lam)
        else:
            kp = 1 if r.k == 1 else (r.k + 3) // 4 * 4  # same layout as the server's buffers
            X = torch.rand(A.cols, kp, device="cuda") * 2 - 1
            Y = torch.empty(A.rows, kp, device="cuda")
            maxe.maxe_spmm(h, X[:, :r.k], Y[:, :r.k], permuted=True)
        bytes_seq += srv.unit_bytes(r) * r.units
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    hbm, src = peaks()
    out = {
        "value": round(sat["gbs"], 3), "unit": "GB/s",
        "config": {"workload": "64 square matrices, rows log-uniform 10k-4M, Poisson(U[5,50]) row lengths, half "
                               "FP32 half BF16 values, R-C permuted, autotuned handles (x-sliced SpMV where faster); "
                               "requests 60% SpMV, 30% SpMM k~U{2..32}, 10% 20-step power iteration; device-memory "
                               "admission cap 60 GB",
                   "requests_per_trace": n, "resident_bytes": srv.resident_bytes,
                   "total_nnz": int(sum(A.nnz for A in mats))},
        "saturation": sat, "loads": at,
        "p50_ms": {f: round(v["p50_ms"], 3) for f, v in at.items()},
        "p99_ms": {f: round(v["p99_ms"], 3) for f, v in at.items()},
        "one_request_at_a_time_bare_launches": {"req_per_s": n / t_seq, "gbs": bytes_seq / t_seq / 1e9,
                                                "what": "requests launched back to back with no scheduler, "
                                                        "no arrivals and no latency accounting"},
        "over_bare": round(sat["req_per_s"] / (n / t_seq), 3),
        "roofline": {"bound": "hbm", "achieved": round(sat["gbs"], 3), "peak": hbm, "unit": "GB/s",
                     "frac": round(sat["gbs"] / hbm, 4), "peak_source": src},
        "gen_s": t_gen, "load_and_tune_s": t_load,
    }
    if unb is not None:
        out["unbatched_server"] = unb
    srv.close()
    return out


def run_serving(args):
    from paper_2308_00106_gb300 import maxe

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    clocks = Clocks(local)
    clocks.start()
    out = serving_measure(args.seed, args.requests)
    clk = clocks.stop()
    out = {"metric": "served p50/p99 latency and GB/s (config: 64 resident permuted matrices, Poisson SpMV/SpMM/"
                     "power-iteration stream, 60 GB cap)", "n_gpus": world, "higher_is_better": True,
           "dtype": "f32/bf16 values, f32 vectors", "data": "synthetic", **out, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def run_spmm_profile(args):
    """SpMM with the rows kernel on a natural-order 5-point Laplacian (grid x
    grid, FP32, k columns): 3 products then 20 timed ones, for ncu captures of
    spmm_rows_kernel (`-s 3 -c 1` takes the first timed launch)."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    maxe.load(build_if_missing=True)
    A = W.laplacian5(args.grid, "f32", "cuda")
    h = maxe.from_csr(A, spmm_rows=True, spmm_rows_pf=args.rows_pf)
    k = args.k
    X = W.matrix_rhs(1, A.cols, k, "f32", "cuda")
    Y = torch.empty(A.rows, k, dtype=torch.float32, device="cuda")
    for _ in range(3):
        maxe.maxe_spmm(h, X, Y, permuted=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        maxe.maxe_spmm(h, X, Y, permuted=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    by = alg_bytes(A.rows, A.cols, A.nnz, 4, 4, 4, k)
    hbm, src = peaks()
    print(json.dumps({"workload": f"5-point Laplacian {args.grid}^2 natural, FP32, k = {k}, rows kernel"
                                  + (" with next-row prefetch" if args.rows_pf else ""),
                      "ms": round(ms, 4), "gbs": round(by / (ms * 1e-3) / 1e9, 1),
                      "frac": round(by / (ms * 1e-3) / 1e9 / hbm, 4), "alg_bytes": by, "peak_source": src}))
    h.close()


def run_laplacian_table(args):
    """5-point Laplacian, n = 4096 (16.8M rows, 83.9M nonzeros): FP64 / FP32 /
    BF16 values x natural / permuted order x SpMM k = 1, 4, 16."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    n = 4096
    hbm, src = peaks()
    rows_out = []
    base = W.laplacian5(n, "f64", "cuda")
    M = N = base.rows
    rperm = maxe.maxe_build_permutation(args.seed, M, 0)
    cperm = maxe.maxe_build_permutation(args.seed, N, 1)
    K = max(10, args.steps // 200)
    clocks = Clocks(local)
    clocks.start()
    for dtype in ("f64", "f32", "bf16"):
        A = base.astype(dtype)
        vb = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
        xb = 8 if dtype == "f64" else 4
        vdt = torch.float64 if dtype == "f64" else torch.float32
        for order in ("natural", "permuted"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = maxe.from_csr(A, rperm, cperm, autotune=True) if order == "permuted" else maxe.from_csr(A, autotune=True)
            torch.cuda.synchronize()
            t_build = time.perf_counter() - t0
            nrp, ncol, nval, _, _ = h.csr()
            vv = nval.cpu()
            vv = vv.view(torch.int16).numpy().view(np.uint16) if dtype == "bf16" else vv.numpy()
            rp_h, col_h = nrp.cpu().numpy(), ncol.cpu().numpy()
            for k in (1, 4, 16):
                kp = (k + 3) // 4 * 4 if k > 1 else 1
                Xb = torch.zeros(N, kp, dtype=vdt, device="cuda")
                Xb[:, :k] = W.matrix_rhs(k, N, k, "f64" if dtype == "f64" else "f32", "cuda")
                X = Xb[:, :k]
                Y = torch.empty(M, kp, dtype=vdt, device="cuda")[:, :k]
                if k == 1:
                    x1 = Xb[:, 0].contiguous()
                    y1 = torch.empty(M, dtype=vdt, device="cuda")
                    step = lambda: maxe.maxe_spmv(h, x1, y1, permuted=True)  # noqa: E731
                else:
                    step = lambda: maxe.maxe_spmm(h, X, Y, permuted=True)  # noqa: E731
                ms, _ = timed_steps(step, K, 3, world, graph_len=5)
                by = alg_bytes(M, N, A.nnz, vb, xb, xb, k)
                gbs = by / (ms * 1e-3) / 1e9
                rows_out.append({"dtype": dtype, "order": order, "k": k, "ms": round(ms, 4), "gbs": round(gbs, 1),
                                 "frac": round(gbs / hbm, 4), "gflops": round(2 * A.nnz * k / (ms * 1e-3) / 1e9, 1),
                                 "items_per_lane": h.items_per_lane(), "xslice": bool(k == 1 and h.xslice()),
                                 "spmm_path": None if k == 1 else (("rows+pf" if h.spmm_rows_prefetch() else "rows")
                                                                   if h.spmm_rows() else
                                                                   "lanes" if h.spmm_lanes() else "passes"),
                                 "build_s": round(t_build, 4)})
            h.close()
    clk = clocks.stop()
    out = {"metric": "SpMV/SpMM GB/s and frac of HBM roofline, 5-point Laplacian on a 4096 x 4096 grid",
           "unit": "GB/s", "peak": hbm, "peak_source": src, "rows": M, "nnz": base.nnz,
           "timing": f"{K} steps, CUDA graph of 5, CUDA events; inputs larger than L2 (matrix >= 0.5 GB)",
           "table": rows_out, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def run_partition_table(args):
    """Equal-rows versus nnz-balanced warp partitions (Section 5: a fixed split by
    equal rows is where random permutation balances the load) and the COO
    product (Section 2), natural and permuted order, FP32 SpMV, on two 1M-row
    matrices: heavy rows clustered at the top (1% of rows x 1000 entries, the
    rest 16) and the power-law matrix.  GB/s counts the CSR's algorithmic bytes
    for all three, so they compare as times."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    hbm, src = peaks()
    K = max(10, args.steps // 100)
    clocks = Clocks(local)
    clocks.start()
    rows_out = []
    for wname, A in (("clustered_heavy_1M", W.clustered_heavy(args.seed, 1 << 20, dtype="f32", device="cuda")),
                     ("powerlaw_1M", W.powerlaw(args.seed, device="cuda"))):
        M, N = A.rows, A.cols
        rperm = maxe.maxe_build_permutation(args.seed, M, 0)
        cperm = maxe.maxe_build_permutation(args.seed, N, 1)
        x = W.vector(1, N, "f32", "cuda")
        for order in ("natural", "permuted"):
            for part in ("nnz_balanced", "equal_rows", "coo"):
                perms = (rperm, cperm) if order == "permuted" else (None, None)
                h = maxe.from_csr(A, *perms, equal_rows=(part == "equal_rows"), coo=(part == "coo"))
                xp = x[cperm.long()] if order == "permuted" else x
                y = torch.empty(M, device="cuda")
                if part == "coo":
                    step = lambda: maxe.maxe_coo_spmv(h, xp, y, permuted=True)  # noqa: E731
                else:
                    step = lambda: maxe.maxe_spmv(h, xp, y, permuted=True)  # noqa: E731
                ms, _ = timed_steps(step, K, 3, world, graph_len=10)
                gbs = alg_bytes(M, N, A.nnz, 4, 4, 4) / (ms * 1e-3) / 1e9  # CSR bytes: COO reads 4 more per entry
                rows_out.append({"matrix": wname, "order": order, "partition": part, "ms": round(ms, 4),
                                 "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)})
                h.close()
        del A
    clk = clocks.stop()
    out = {"metric": "FP32 SpMV GB/s, equal-rows vs nnz-balanced warp partition vs COO, natural vs permuted",
           "unit": "GB/s", "peak": hbm, "peak_source": src,
           "timing": f"{K} steps, CUDA graph of 10, CUDA events; inputs larger than L2",
           "table": rows_out, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def run_shuffle_table(args):
    """The four randomisation formats of the appendix (R, RC, G-R, G-C) beside the
    natural order: 64x64-grid entropy (Section 4), the spread of the 8x8
    hierarchical entropy map (Section 5), one-time preprocessing time, and FP32
    SpMV under the nnz-balanced and the equal-rows warp partitions."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    hbm, src = peaks()
    K = max(10, args.steps // 100)
    clocks = Clocks(local)
    clocks.start()
    rows_out = []
    mats = (("blockdiag_4096", lambda: W.blockdiag(args.seed, dtype="f32", device="cuda")),
            ("clustered_heavy_1M", lambda: W.clustered_heavy(args.seed, 1 << 20, dtype="f32", device="cuda")),
            ("powerlaw_1M", lambda: W.powerlaw(args.seed, device="cuda")))
    for wname, make in mats:
        A = make()
        M, N = A.rows, A.cols
        x = W.vector(1, N, "f32", "cuda")
        for fmt in ("natural", "R", "RC", "G-R", "G-C"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if fmt in ("R", "RC"):
                rperm = maxe.maxe_build_permutation(args.seed, M, 0)
                cperm = maxe.maxe_build_permutation(args.seed, N, 1) if fmt == "RC" else None
            elif fmt in ("G-R", "G-C"):
                rperm, cperm = maxe.gradient_perms(A, args.seed, columns=(fmt == "G-C"))
            else:
                rperm = cperm = None
            handles = {"nnz_balanced": maxe.from_csr(A, rperm, cperm)}
            torch.cuda.synchronize()
            t_pre = time.perf_counter() - t0
            handles["equal_rows"] = maxe.from_csr(A, rperm, cperm, equal_rows=True)
            h = handles["nnz_balanced"]
            H, cnt = maxe.maxe_nnz_entropy(h, 64, 64)
            lv = maxe.maxe_entropy_levels(cnt, 8).cpu().numpy()
            xp = x[cperm.long()] if cperm is not None else x
            row = {"matrix": wname, "format": fmt, "entropy_64x64": round(H, 4),
                   "map8_min": round(float(lv.min()), 4), "map8_max": round(float(lv.max()), 4),
                   "preprocess_ms": round(t_pre * 1e3, 3)}
            for part, hh in handles.items():
                y = torch.empty(M, device="cuda")
                step = lambda: maxe.maxe_spmv(hh, xp, y, permuted=True)  # noqa: E731
                ms, _ = timed_steps(step, K, 3, world, graph_len=10)
                gbs = alg_bytes(M, N, A.nnz, 4, 4, 4) / (ms * 1e-3) / 1e9
                row[part] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)}
                hh.close()
            rows_out.append(row)
        del A
    clk = clocks.stop()
    out = {"metric": "entropy and FP32 SpMV GB/s per randomisation format (natural, R, RC, G-R, G-C)",
           "unit": "GB/s", "peak": hbm, "peak_source": src,
           "timing": f"{K} steps, CUDA graph of 10, CUDA events; preprocess = permutations + permute_csr, host clock",
           "table": rows_out, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))


def by_dtype_measure(base, rperm, cperm, K, warmup, world, dtypes=("f64", "bf16")):
    """The headline matrix with its values stored in other types (a8): the same
    launch configuration (autotuned handles, vectors in the permuted space),
    permuted and natural order.  Returns {dtype: {order: record}} and, per
    (dtype, order), the original-space product y = A x of the same handle for
    the oracle check (the same kernel and values, x gathered and y scattered)."""
    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    hbm, _ = peaks()
    M, N, Z = base.rows, base.cols, base.nnz
    out, ys = {}, {}  # ys[(dtype, order)] = (x, y = A x): the oracle check reuses the same x
    for dt in dtypes:
        A = base.astype(dt)
        vb = {"f64": 8, "f32": 4, "bf16": 2}[dt]
        xb = 8 if dt == "f64" else 4
        by = alg_bytes(M, N, Z, vb, xb, xb)
        x = W.vector(1, N, "f64" if dt == "f64" else "f32", "cuda")
        out[dt] = {}
        for order, perms in (("permuted", (rperm, cperm)), ("plain", (None, None))):
            h = maxe.from_csr(A, *perms, autotune=True)
            xp = maxe.maxe_permute_gather(cperm, x) if order == "permuted" else x
            y = torch.empty(M, dtype=x.dtype, device="cuda")
            ms, _ = timed_steps(lambda: maxe.maxe_spmv(h, xp, y, permuted=True), K, warmup, world, 50)
            gbs = by / (ms * 1e-3) / 1e9
            out[dt][order] = {"gbs": round(gbs, 1), "frac": round(gbs / hbm, 4), "us": round(ms * 1e3, 2),
                              "alg_bytes": by, "kernel": ("x-sliced" + (" pairs" if h.xslice_pairs() else ""))
                              if h.xslice() else "csr"}
            ys[(dt, order)] = (x.cpu().double().numpy(), maxe.maxe_spmv(h, x).cpu().numpy())
            h.close()
        del A
    return out, ys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["maxe", "reference"], default="maxe")
    ap.add_argument("--workload", choices=["powerlaw", "laplacian", "blockdiag", "clustered", "batched", "serving",
                                           "laplacian-table", "partition-table", "shuffle-table", "spmm-profile"],
                    default="powerlaw")
    ap.add_argument("--requests", type=int, default=1500, help="requests per serving trace")
    ap.add_argument("--grid", type=int, default=2048, help="spmm-profile: Laplacian grid side")
    ap.add_argument("--k", type=int, default=16, help="spmm-profile: right-hand sides")
    ap.add_argument("--rows-pf", action="store_true", help="spmm-profile: rows kernel with its next-row prefetch")
    ap.add_argument("--batch-count", type=int, default=256, help="matrices of the batched workload")
    ap.add_argument("--no-tune", action="store_true", help="batched workload: default batch plans, no autotuning")
    ap.add_argument("--e2e-streams", type=int, default=3,
                    help="streams the end-to-end steps rotate over (each with its own host and device buffers)")
    ap.add_argument("--items-per-lane", choices=["auto", "8", "16"], default="auto",
                    help="SpMV kernel variant: autotuned per handle, or fixed")
    ap.add_argument("--xslice", action="store_true",
                    help="SpMV on the x-sliced form for both handles (no autotuning); for profiling that kernel")
    ap.add_argument("--seed", type=int, default=2308)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-workers", type=int, default=1,
                    help="reference arm: split the oracle's product into this many equal-row ranges on threads "
                         "(the paper's parallel CPU CSR), timed for the natural and the permuted matrix")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph-len", type=int, default=50)
    ap.add_argument("--seeds", type=int, default=32, help="permutation seeds of the min/mean/max sweep (0: skip)")
    ap.add_argument("--profile", action="store_true",
                    help="no timing: 3 permuted then 3 plain SpMV launches (for an ncu capture)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: leave out the by-value-type, serving and batched sections")
    ap.add_argument("--serve-requests", type=int, default=400, help="requests per trace of the serving section")
    ap.add_argument("--record-profile", nargs=4, metavar=("CSV", "KERNEL", "LAUNCH", "COMMAND"),
                    help="write profiles/<record>.json from an ncu raw CSV export (no GPU needed)")
    args = ap.parse_args()
    if args.e2e_streams < 1:
        ap.error("--e2e-streams must be at least 1")
    if args.record_profile:
        csv_path, kernel, launch, command = args.record_profile
        print(json.dumps(record_profile(csv_path, kernel, int(launch), command, args.workload)))
        return
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "shuffle-table":
        return run_shuffle_table(args)
    if args.workload == "partition-table":
        return run_partition_table(args)
    if args.workload == "spmm-profile":
        return run_spmm_profile(args)
    if args.workload == "laplacian-table":
        return run_laplacian_table(args)

    from paper_2308_00106_gb300 import maxe
    from paper_2308_00106_gb300 import workloads as W

    rank, world, local = dist_setup(args)
    maxe.load(build_if_missing=(rank == 0))
    A, dtype, desc = make_workload(args.workload, args.seed, "cuda")
    M, N, Z = A.rows, A.cols, A.nnz
    vb = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
    xb = 8 if dtype == "f64" else 4
    vdt = torch.float64 if dtype == "f64" else torch.float32

    # ---- one-time preprocessing (Section 3: permutation; Section 4: entropy)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record()
    rperm = maxe.maxe_build_permutation(args.seed, M, 0)
    cperm = maxe.maxe_build_permutation(args.seed, N, 1)
    ev[1].record()
    tune = args.items_per_lane == "auto" and not args.xslice
    i16 = args.items_per_lane == "16"
    hP = maxe.from_csr(A, rperm, cperm, autotune=tune, items16=i16, xslice=args.xslice)
    ev[2].record()
    hN = maxe.from_csr(A, autotune=tune, items16=i16, xslice=args.xslice)
    ev[3].record()
    torch.cuda.synchronize()
    t_perm, t_pcsr = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    t0 = time.perf_counter()
    H_perm, _ = maxe.maxe_nnz_entropy(hP, 64, 64, counts=False)
    t_ent = (time.perf_counter() - t0) * 1e3
    H_plain, _ = maxe.maxe_nnz_entropy(hN, 64, 64, counts=False)

    x = W.vector(1, N, "f64" if dtype == "f64" else "f32", "cuda")
    xp = maxe.maxe_permute_gather(cperm, x)
    yP = torch.empty(M, dtype=vdt, device="cuda")
    yN = torch.empty(M, dtype=vdt, device="cuda")
    yF = torch.empty(M, dtype=vdt, device="cuda")

    def step_perm():
        maxe.maxe_spmv(hP, xp, yP, permuted=True)

    def step_plain():
        maxe.maxe_spmv(hN, x, yN, permuted=True)

    def step_full():
        maxe.maxe_spmv(hP, x, yF)

    if args.profile:
        for f in (step_perm, step_perm, step_perm, step_plain, step_plain, step_plain):
            f()
        torch.cuda.synchronize()
        print(json.dumps({"profile": "done", "rows": M, "nnz": Z}))
        return

    clocks = Clocks(local)
    clocks.start()
    ms_perm, graphed = timed_steps(step_perm, args.steps, args.warmup, world, args.graph_len)
    clk = clocks.stop()
    ms_plain, _ = timed_steps(step_plain, args.steps, args.warmup, world, args.graph_len)
    ms_full, _ = timed_steps(step_full, max(args.steps // 4, 1), args.warmup, world, args.graph_len)
    fl_perm = flushed_launch_ms(step_perm, reps=200)
    fl_plain = flushed_launch_ms(step_plain, reps=200)
    seeds = seed_sweep(A, x, args, world, tune) if args.seeds > 0 else None

    bytes_step = alg_bytes(M, N, Z, vb, xb, xb)
    gbs = bytes_step / (ms_perm * 1e-3) / 1e9  # one replica; the job's value is job_rate over all ranks
    gbs_plain = bytes_step / (ms_plain * 1e-3) / 1e9
    hbm, src = peaks()

    nrp, ncol, nval, _, _ = hP.csr()

    # ---- end to end through the public API with host buffers: every step is one
    # maxe_spmv_host call that copies its x' from pinned host memory, runs the
    # product and copies y' back; steps rotate over --e2e-streams streams with
    # their own buffers, so one step's copies overlap the other steps' products
    # (with two, a stream's D2H of one step and H2D of its next step must both
    # fit in the time of one product)
    K_e2e = max(args.steps // 4, 2)
    e2e_streams = [torch.cuda.Stream() for _ in range(args.e2e_streams)]
    e2e_bufs = [(xp.cpu().pin_memory(), torch.empty_like(xp), torch.empty(M, dtype=vdt, device="cuda"),
                 torch.empty(M, dtype=vdt).pin_memory()) for _ in e2e_streams]

    def step_e2e(k):
        st = e2e_streams[k % len(e2e_streams)]
        xh, xd, yd, yh = e2e_bufs[k % len(e2e_streams)]
        maxe.maxe_spmv_host(hP, xh, yh, xd, yd, permuted=True, stream=st)

    host_e2e = []
    ms_e2e = timed_streams(step_e2e, e2e_streams, K_e2e, args.warmup, world, host_e2e)
    for b in e2e_bufs[1:]:
        np.testing.assert_array_equal(e2e_bufs[0][3].numpy(), b[3].numpy())  # same product on every stream
    if not torch.equal(e2e_bufs[0][3].cuda(), yP):
        raise SystemExit("end-to-end result differs from the timed device result")

    kern = "spmv_xslice_kernel" if hP.xslice() else "spmm_warp_kernel"
    traffic = traffic_from_record(kern)

    # ---- the rest of the metric: other value types, the served and batched forms
    by_dtype, by_dtype_y, serving, batched = None, {}, None, None
    if not args.no_extras and args.workload == "powerlaw":
        K_x = max(min(args.steps, 2000), 2)
        by_dtype, by_dtype_y = by_dtype_measure(A, rperm, cperm, K_x, args.warmup, world)
        by_dtype["f32"] = {"permuted": {"gbs": round(gbs, 1), "frac": round(gbs / hbm, 4),
                                        "us": round(ms_perm * 1e3, 2), "alg_bytes": bytes_step,
                                        "kernel": ("x-sliced" + (" pairs" if hP.xslice_pairs() else ""))
                                        if hP.xslice() else "csr"},
                           "plain": {"gbs": round(gbs_plain, 1), "frac": round(gbs_plain / hbm, 4),
                                     "us": round(ms_plain * 1e3, 2), "alg_bytes": bytes_step,
                                     "kernel": "x-sliced" if hN.xslice() else "csr"}}
        by_dtype_y[("f32", "permuted")] = (x.cpu().double().numpy(), maxe.maxe_spmv(hP, x).cpu().numpy())
        by_dtype_y[("f32", "plain")] = (x.cpu().double().numpy(), maxe.maxe_spmv(hN, x).cpu().numpy())
        serving = serving_measure(args.seed, args.serve_requests, loads=(0.5, 0.8), unbatched=False)
        batched = batched_measure(args.seed, 256, max(1, min(args.steps // 10, 5)), args.warmup, world, tune=True)

    out = {
        "metric": METRIC, "value": round(job_rate(bytes_step, ms_perm, world) / 1e9, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_perm, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": desc, "rows": M, "nnz": Z, "seed": args.seed,
                   "variant": "permuted R-C (rows and columns), vectors in permuted space",
                   "l2": "inputs larger than L2 (matrix %.0f MB > 129 MB); x', y' stay L2-resident across steps"
                         % (bytes_step / 1e6),
                   "timing": (f"{args.steps} steps as CUDA graph replays of {min(args.graph_len, args.steps)} "
                              f"steps" if graphed else f"{args.steps} eager launch(es)")
                             + ", CUDA events on the launching stream, max over ranks",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "plain": {"value": round(gbs_plain * world, 3), "unit": "GB/s", "ms_per_step": ms_plain,
                  "frac": round(gbs_plain / hbm, 4)},
        "gflops": {"permuted": round(2 * Z * world / (ms_perm * 1e-3) / 1e9, 2),
                   "plain": round(2 * Z * world / (ms_plain * 1e-3) / 1e9, 2), "what": "2 nnz / time"},
        "permuted_over_plain": round(ms_plain / ms_perm, 4),
        "kernel_variant": {"permuted_items_per_lane": hP.items_per_lane(), "plain_items_per_lane": hN.items_per_lane(),
                           "permuted_xslice": hP.xslice(), "plain_xslice": hN.xslice(),
                           "permuted_xslice_pairs": hP.xslice_pairs(), "permuted_stream_prefetch": hP.xslice_ahead()},
        "flushed_l2_launch_ms": {"permuted": fl_perm, "plain": fl_plain, "what": "median of 200 launches, "
                                 "a 256 MB write before each"},
        "seeds": seeds,
        "full_path": {"value": round(bytes_step / (ms_full * 1e-3) / 1e9, 3), "unit": "GB/s",
                      "ms_per_step": ms_full, "what": "y = A x in the original space: x gather + SpMV with fused "
                                                      "y scatter (algorithmic bytes of the product only)"},
        "preprocess_ms": {"build_permutation_rows_and_cols": t_perm, "permute_csr_with_autotune": t_pcsr,
                          "nnz_entropy_64x64": t_ent},
        "entropy_64x64": {"plain": H_plain, "permuted": H_perm, "max": 12.0},
        "roofline": {"bound": "hbm", "achieved": round(gbs, 3), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 4), "traffic": traffic, "peak_source": src,
                     "bytes_per_launch": bytes_step, "kernel": kern},
        "e2e": {"value": round(job_rate(bytes_step, ms_e2e, world) / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": N * xb, "d2h_bytes_per_step": M * xb, "ms_per_step": ms_e2e,
                "host_enqueue_ms_per_step": round(host_e2e[0], 5),
                "what": "per step: one maxe_spmv_host call (H2D of x' from pinned memory, y' = A' x', D2H of y'); "
                        f"steps rotate over {args.e2e_streams} streams",
                "note": "products on different streams overlap one kernel's last CTAs with the next one's first, "
                        "so this can match or pass `value`, which replays the products on one stream"},
        "gpu_launches": args.steps,
        "clocks": clk,
        **({"by_dtype": by_dtype} if by_dtype else {}),
        **({"serving": serving} if serving else {}),
        **({"batched": batched} if batched else {}),
        "context": "paper: ~15% gain from randomization on AMD GPU-CPU systems (FP64, rocSPARSE); context only",
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, reps, y_cpu = cpu_baseline(tuple(a.cpu().numpy() if a.dtype != torch.bfloat16 else
                                                a.cpu().view(torch.int16).numpy() for a in (nrp, ncol, nval)),
                                          xp.cpu().double().numpy(), W.DTYPE_CODE[dtype], args.cpu_seconds)
        got = yP.cpu().double().numpy()
        out["cpu_baseline"] = {"value": round(bytes_step / t_cpu / 1e9, 4), "unit": "GB/s", "cores": 1,
                               "kind": "oracle", "sample": f"full permuted matrix, {reps} products, FP64 oracle",
                               "host": host_info(),
                               "rel_l2_gpu_vs_oracle": float(np.linalg.norm(got - y_cpu) /
                                                             max(np.linalg.norm(y_cpu), 1e-300))}
        if by_dtype:
            # every value type and order against the FP64 oracle on its stored
            # values, all rows (y = A x through each handle, original space)
            import oracle
            rp0, co0 = A.rowptr.cpu().numpy(), A.col.cpu().numpy()
            for dt in by_dtype:
                vv = A.astype(dt).val.cpu()
                vv = vv.view(torch.int16).numpy().view(np.uint16) if dt == "bf16" else vv.numpy()
                for order in by_dtype[dt]:
                    xd, yy = by_dtype_y[(dt, order)]
                    ref = oracle.spmv(M, rp0, co0, vv, W.DTYPE_CODE[dt], xd)
                    by_dtype[dt][order]["rel_l2_vs_oracle"] = float(np.linalg.norm(yy.astype(np.float64) - ref) /
                                                                    max(np.linalg.norm(ref), 1e-300))
    if rank == 0:
        print(json.dumps(out))
    hP.close()
    hN.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
