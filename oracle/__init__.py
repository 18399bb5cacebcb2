"""CPU oracle for the max_E SpMV hot path (arXiv 2308.00106).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The product path (the CUDA library and
its binding) never imports this package, and this package never imports the
product. The arithmetic lives in ``oracle.c`` (plain single-threaded C, FP64);
this module only compiles it with gcc on first use and marshals numpy arrays.

Each wrapper names the passage of the paper it states:
  build_permutation / invert_permutation / gather / scatter  -- Section 3 and Eq. 1
  permute_csr                                                  -- Eq. 1 on CSR (Section 2)
  nnz_entropy                                                  -- Section 4, entropy equation
  entropy_levels                                               -- Section 5, hierarchical 2-D entropy
  nnz_histogram / gradient_permutation                         -- Section 5 and appendix, gradient shuffles
  spmv / spmm / spmv_rows                                      -- Section 2, CSR product
  coo_spmv / csr_to_coo_rows                                   -- Section 2, COO product
  power_iteration                                              -- not in the paper (serving reference)

Parity of the paper's printed entropies (8.39, 8.41, 11.27, ...) is unpinned:
the matrices and the histogram binning they were measured with are not given.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F64, F32, BF16 = 0, 1, 2

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_key.restype = ctypes.c_uint64
            lib.orc_key.argtypes = [ctypes.c_uint64, _I32, _I64]
            lib.orc_build_permutation.argtypes = [ctypes.c_uint64, _I32, _I32, _P]
            lib.orc_invert_permutation.argtypes = [_P, _I32, _P]
            lib.orc_gather.argtypes = [_P, _I32, _P, _P]
            lib.orc_scatter.argtypes = [_P, _I32, _P, _P]
            lib.orc_permute_csr.argtypes = [_I32, _I32, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]
            lib.orc_nnz_entropy.restype = ctypes.c_double
            lib.orc_nnz_entropy.argtypes = [_I32, _I32, _P, _P, _I32, _I32, ctypes.c_double, _P]
            lib.orc_spmv.argtypes = [_I32, _P, _P, _P, ctypes.c_int, _P, _P]
            lib.orc_entropy_levels.argtypes = [_P, _I32, _I32, _I32, ctypes.c_double, _P]
            lib.orc_coo_spmv.argtypes = [_I32, _I64, _P, _P, _P, ctypes.c_int, _P, _P]
            lib.orc_csr_to_coo_rows.argtypes = [_I32, _P, _P]
            lib.orc_nnz_histogram.argtypes = [_I32, _I32, _P, _P, _I32, _P]
            lib.orc_gradient_permutation.argtypes = [_P, _I32, ctypes.c_uint64, _I32, _P, _P]
            lib.orc_spmm.argtypes = [_I32, _P, _P, _P, ctypes.c_int, _I32, _P, _I64, _P, _I64]
            lib.orc_spmv_rows.argtypes = [_P, _P, _P, ctypes.c_int, _P, _P, _I64, _P]
            lib.orc_power_iteration.restype = ctypes.c_double
            lib.orc_power_iteration.argtypes = [_I32, _P, _P, _P, ctypes.c_int, _P, _I32, _P, _P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _vals(val: np.ndarray, dtype: int) -> np.ndarray:
    want = {F64: np.float64, F32: np.float32, BF16: np.uint16}[dtype]
    if val.dtype == np.int16 and dtype == BF16:
        val = val.view(np.uint16)
    if val.dtype != want:
        raise TypeError(f"values must be {np.dtype(want)} for dtype code {dtype}, got {val.dtype}")
    return np.ascontiguousarray(val)


def key(seed: int, tag: int, i: int) -> int:
    """Output number 2*i+tag+1 of SplitMix64 seeded with `seed` (Section 3 reading)."""
    return int(_load().orc_key(seed & (2**64 - 1), tag, i))


def build_permutation(seed: int, n: int, tag: int) -> np.ndarray:
    """perm[new] = old: indices sorted by (key, index) (Section 3; Eq. 1)."""
    perm = np.empty(max(n, 0), dtype=np.int32)
    rc = _load().orc_build_permutation(seed & (2**64 - 1), n, tag, _ptr(perm))
    if rc != 0:
        raise ValueError("build_permutation failed")
    return perm


def invert_permutation(perm) -> np.ndarray:
    perm = _i32(perm)
    inv = np.empty_like(perm)
    if _load().orc_invert_permutation(_ptr(perm), perm.size, _ptr(inv)) != 0:
        raise ValueError("not a permutation")
    return inv


def gather(perm, x) -> np.ndarray:
    """x' = P_c^{-1} x, i.e. out[i] = x[perm[i]] (Eq. 1)."""
    perm, x = _i32(perm), _f64(x)
    out = np.empty(perm.size, dtype=np.float64)
    _load().orc_gather(_ptr(perm), perm.size, _ptr(x), _ptr(out))
    return out


def scatter(perm, y) -> np.ndarray:
    """y = P_r^{-1} y', i.e. out[perm[i]] = y'[i] (Eq. 1)."""
    perm, y = _i32(perm), _f64(y)
    out = np.empty(perm.size, dtype=np.float64)
    _load().orc_scatter(_ptr(perm), perm.size, _ptr(y), _ptr(out))
    return out


def permute_csr(M: int, N: int, rowptr, col, val, dtype: int, rperm=None, cperm=None):
    """A' = P_r A P_c in CSR with ascending columns; values copied bit for bit (Eq. 1)."""
    rowptr, col, val = _i32(rowptr), _i32(col), _vals(val, dtype)
    rp = None if rperm is None else _i32(rperm)
    cp = None if cperm is None else _i32(cperm)
    ro = np.empty(M + 1, dtype=np.int32)
    co = np.empty(col.size, dtype=np.int32)
    vo = np.empty_like(val)
    rc = _load().orc_permute_csr(M, N, _ptr(rowptr), _ptr(col), _ptr(val), dtype, _ptr(rp), _ptr(cp),
                                 _ptr(ro), _ptr(co), _ptr(vo))
    if rc != 0:
        raise ValueError("permute_csr: bad permutation")
    return ro, co, vo


def nnz_entropy(M: int, N: int, rowptr, col, gr: int, gc: int, base: float = 2.0):
    """(H, counts[gr, gc]) for the block-grid histogram of the nonzeros (Section 4)."""
    if not (1 <= gr <= M and 1 <= gc <= N):
        raise ValueError("grid must satisfy 1 <= gr <= M, 1 <= gc <= N")
    rowptr, col = _i32(rowptr), _i32(col)
    counts = np.empty(gr * gc, dtype=np.int64)
    H = _load().orc_nnz_entropy(M, N, _ptr(rowptr), _ptr(col), gr, gc, float(base), _ptr(counts))
    return float(H), counts.reshape(gr, gc)


def entropy_levels(counts, L: int, base: float = 2.0) -> np.ndarray:
    """L x L map of block entropies of a (gr, gc) count grid (Section 5, hierarchical 2-D entropy)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    gr, gc = counts.shape
    if not (1 <= L <= gr and L <= gc):
        raise ValueError("need 1 <= L <= gr, gc")
    out = np.empty(L * L, dtype=np.float64)
    _load().orc_entropy_levels(_ptr(counts), gr, gc, L, float(base), _ptr(out))
    return out.reshape(L, L)


def nnz_histogram(M: int, N: int, rowptr, col, axis: int) -> np.ndarray:
    """Entries per row (axis 0) or per column (axis 1) (Section 5, appendix)."""
    rowptr, col = _i32(rowptr), _i32(col)
    h = np.empty(M if axis == 0 else N, dtype=np.int32)
    _load().orc_nnz_histogram(M, N, _ptr(rowptr), _ptr(col), int(axis), _ptr(h))
    return h


def gradient_permutation(hist, seed: int, tag: int):
    """(perm, pivot): cut at the steepest histogram gradient, riffle, permute each
    half of the shuffled deck at random (appendix, gradient-based permutations)."""
    hist = _i32(hist)
    perm = np.empty(hist.size, dtype=np.int32)
    pivot = ctypes.c_int32(-1)
    if _load().orc_gradient_permutation(_ptr(hist), hist.size, seed & (2**64 - 1), tag, _ptr(perm),
                                        ctypes.byref(pivot)) != 0:
        raise ValueError("gradient_permutation failed")
    return perm, int(pivot.value)


def spmv(M: int, rowptr, col, val, dtype: int, x) -> np.ndarray:
    """y = A x in FP64 over the stored values, stored order (Section 2)."""
    rowptr, col, val, x = _i32(rowptr), _i32(col), _vals(val, dtype), _f64(x)
    y = np.empty(M, dtype=np.float64)
    _load().orc_spmv(M, _ptr(rowptr), _ptr(col), _ptr(val), dtype, _ptr(x), _ptr(y))
    return y


def coo_spmv(M: int, row, col, val, dtype: int, x) -> np.ndarray:
    """y = A x over COO triplets in stored order, any order allowed (Section 2)."""
    row, col, val, x = _i32(row), _i32(col), _vals(val, dtype), _f64(x)
    y = np.empty(M, dtype=np.float64)
    _load().orc_coo_spmv(M, row.size, _ptr(row), _ptr(col), _ptr(val), dtype, _ptr(x), _ptr(y))
    return y


def csr_to_coo_rows(M: int, rowptr) -> np.ndarray:
    """Row index of every stored entry of a CSR matrix (its COO form, Section 2)."""
    rowptr = _i32(rowptr)
    row = np.empty(int(rowptr[M]) if M > 0 else 0, dtype=np.int32)
    _load().orc_csr_to_coo_rows(M, _ptr(rowptr), _ptr(row))
    return row


def spmm(M: int, rowptr, col, val, dtype: int, X) -> np.ndarray:
    """Y = A X for row-major X (N x k) in FP64 (Section 2, k right-hand sides)."""
    rowptr, col, val = _i32(rowptr), _i32(col), _vals(val, dtype)
    X = _f64(X)
    k = X.shape[1]
    Y = np.empty((M, k), dtype=np.float64)
    _load().orc_spmm(M, _ptr(rowptr), _ptr(col), _ptr(val), dtype, k, _ptr(X), k, _ptr(Y), k)
    return Y


def spmv_rows(rowptr, col, val, dtype: int, x, rows) -> np.ndarray:
    """y_i for the listed rows only (Section 2), for one-by-one checks of large cases."""
    rowptr, col, val, x = _i32(rowptr), _i32(col), _vals(val, dtype), _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(rows.size, dtype=np.float64)
    _load().orc_spmv_rows(_ptr(rowptr), _ptr(col), _ptr(val), dtype, _ptr(x), _ptr(rows), rows.size, _ptr(y))
    return y


def power_iteration(M: int, rowptr, col, val, dtype: int, v0, steps: int, history: bool = False):
    """lambda, v after `steps` normalised products v <- A v / ||A v|| (not in the paper)."""
    rowptr, col, val, v0 = _i32(rowptr), _i32(col), _vals(val, dtype), _f64(v0)
    v = np.empty(M, dtype=np.float64)
    hist = np.empty(max(steps, 1), dtype=np.float64) if history else None
    lam = _load().orc_power_iteration(M, _ptr(rowptr), _ptr(col), _ptr(val), dtype, _ptr(v0), steps,
                                      _ptr(v), _ptr(hist))
    if history:
        return float(lam), v, hist[:steps]
    return float(lam), v
