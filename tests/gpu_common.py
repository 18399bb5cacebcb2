"""Helpers shared by the GPU parity tests (inputs, oracle calls, tolerances)."""
import numpy as np
import torch

import oracle
from paper_2308_00106_gb300 import workloads as W

# relative L2 error bounds against the FP64 oracle on the stored values
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 2e-3}


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(got - ref)
    n = np.linalg.norm(ref)
    return float(d / n) if n > 0 else float(d)


def code(dtype: str) -> int:
    return W.DTYPE_CODE[dtype]


def vec_dtype(dtype: str):
    return torch.float64 if dtype == "f64" else torch.float32


def edge_matrix(kind: str, dtype: str = "f32", seed: int = 0) -> W.CSR:
    """Small matrices that hit the corner cases of the chunked kernels."""
    g = np.random.default_rng(seed)
    if kind == "one":
        return W.from_lengths(seed, [1], 1, dtype)
    if kind == "empty_nnz":
        return W.from_lengths(seed, [0] * 37, 11, dtype)
    if kind == "ragged":  # several 2048-entry chunks plus a ragged tail
        return W.from_lengths(seed, g.integers(0, 60, 3000), 5000, dtype)
    if kind == "empty_runs":  # long runs of empty rows (more rows per chunk than the smem slice holds)
        lengths = np.zeros(20000, dtype=np.int64)
        lengths[::997] = g.integers(1, 40, lengths[::997].size)
        lengths[5000:5100] = 3
        return W.from_lengths(seed, lengths, 3000, dtype)
    if kind == "unit_rows":  # 1 entry per row: > kRowCap rows per chunk
        return W.from_lengths(seed, np.ones(9000, dtype=np.int64), 9000, dtype)
    if kind == "long_rows":  # rows longer than a chunk and than the bucket sort tile
        lengths = g.integers(0, 30, 400)
        lengths[[3, 50, 51, 399]] = [5000, 2049, 2048, 20000]
        lengths[200] = 70000
        return W.from_lengths(seed, lengths, 80000, dtype)
    if kind == "rect_wide":
        return W.from_lengths(seed, g.integers(0, 50, 700), 50000, dtype)
    if kind == "rect_tall":
        return W.from_lengths(seed, g.integers(0, 9, 20000), 40, dtype)
    raise KeyError(kind)


EDGE_KINDS = ["one", "empty_nnz", "ragged", "empty_runs", "unit_rows", "long_rows", "rect_wide", "rect_tall"]


def oracle_permuted(A: W.CSR, rperm, cperm):
    rp, co, va = A.numpy()
    r = None if rperm is None else rperm.cpu().numpy()
    c = None if cperm is None else cperm.cpu().numpy()
    return oracle.permute_csr(A.rows, A.cols, rp, co, va, code(A.dtype), r, c)


def handle_arrays(h):
    rp, col, val, rperm, cperm = h.csr()
    v = val.cpu()
    if val.dtype == torch.bfloat16:
        v = v.view(torch.int16).numpy().view(np.uint16)
    else:
        v = v.numpy()
    return rp.cpu().numpy(), col.cpu().numpy(), v
