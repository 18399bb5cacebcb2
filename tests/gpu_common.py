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


# unit roundoff of the accumulation: FP64 for FP64 values, FP32 otherwise
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24}
# BF16 values are decoded exactly and accumulated in FP32, so a correct kernel's
# error is FP32 rounding: a regression bound much tighter than the 2e-3 contract
BF16_TIGHT = 1e-5


def abs_values(va: np.ndarray, dtype: str) -> np.ndarray:
    """|values| in the stored encoding (BF16: sign bit cleared)."""
    if dtype == "bf16":
        return (va.view(np.uint16) & np.uint16(0x7FFF)).astype(np.uint16)
    return np.abs(va)


def check_all_rows(y, rp, co, va, dtype: str, x, what=""):
    """Every row of y = A x against the FP64 oracle on the stored values:
    relative L2 within TOL (and BF16_TIGHT for BF16 values), and per row
    |y_i - y_i*| <= (2 n_i + 2) u sum_j |a_ij x_j| -- the rounding bound of any
    order of the row's n_i products and at most 2 n_i + 1 additions (entries,
    partial sums of split rows and halves), u the accumulation's unit roundoff.
    So one wrong row cannot hide in the norm."""
    y = np.asarray(y, dtype=np.float64)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    M = len(rp) - 1
    ref = oracle.spmv(M, rp, co, va, code(dtype), x)
    mag = oracle.spmv(M, rp, co, abs_values(va, dtype), code(dtype), np.abs(x))
    n = np.diff(np.asarray(rp, dtype=np.int64))
    bound = (2 * n + 2) * UNIT[dtype] * mag * 1.01
    bad = np.abs(y - ref) > bound
    assert not bad.any(), (what, int(bad.sum()), int(np.argmax(bad)))
    err = rel_l2(y, ref)
    assert err <= TOL[dtype], (what, err)
    if dtype == "bf16":
        assert err <= BF16_TIGHT, (what, err)
    return err


def check_all_rows_spmm(Y, rp, co, va, dtype: str, X, what=""):
    """check_all_rows for Y = A X with k columns (every row and column), from
    the oracle's SpMM of A X and of |A| |X|."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim == 1:
        return check_all_rows(Y, rp, co, va, dtype, X, what)
    M = len(rp) - 1
    ref = oracle.spmm(M, rp, co, va, code(dtype), X)
    mag = oracle.spmm(M, rp, co, abs_values(va, dtype), code(dtype), np.abs(X))
    n = np.diff(np.asarray(rp, dtype=np.int64))[:, None]
    bound = (2 * n + 2) * UNIT[dtype] * mag * 1.01
    bad = np.abs(Y - ref) > bound
    assert not bad.any(), (what, int(bad.sum()), np.unravel_index(int(np.argmax(bad)), bad.shape))
    err = rel_l2(Y, ref)
    assert err <= TOL[dtype], (what, err)
    if dtype == "bf16":
        assert err <= BF16_TIGHT, (what, err)
    return err
