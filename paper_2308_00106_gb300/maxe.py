"""Thin ctypes binding of libmaxe.so (C ABI in include/maxe.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Torch provides device memory (its caching allocator is handed
to the library as a ``maxe_allocator``) and the current CUDA stream.  There is
no CPU fallback: if the library is missing or no GPU is visible, these calls
raise.

Function names follow the C entry points.  Permutations use perm[new] = old
(Eq. 1 of arXiv 2308.00106):  A' = P_r A P_c,  x' = x[cperm],  y[rperm] = y'.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

import torch

from . import build as _build

MAXE_OK, MAXE_ERR_INVALID, MAXE_ERR_OOM, MAXE_ERR_CUDA, MAXE_ERR_TIMEOUT, MAXE_ERR_UNSUPPORTED = range(6)
MAXE_F64, MAXE_F32, MAXE_BF16 = 0, 1, 2
MAXE_VEC_PERMUTED = 0x1
MAXE_VALIDATE = 0x2
MAXE_AUTOTUNE = 0x4
MAXE_ITEMS16 = 0x8
MAXE_SPMM_LANES = 0x10
MAXE_EQUAL_ROWS = 0x20
MAXE_COO = 0x40
MAXE_XSLICE = 0x80
MAXE_XS_PAIRS = 0x100
MAXE_XS_SINGLE = 0x200
MAXE_SPMM_ROWS = 0x400
MAXE_SPMM_ROWS_PF = 0x800

DTYPE_CODE = {"f64": MAXE_F64, "f32": MAXE_F32, "bf16": MAXE_BF16}
VAL_TORCH = {MAXE_F64: torch.float64, MAXE_F32: torch.float32, MAXE_BF16: torch.bfloat16}
VEC_TORCH = {MAXE_F64: torch.float64, MAXE_F32: torch.float32, MAXE_BF16: torch.float32}

EXPORTS = [
    "maxe_build_permutation", "maxe_invert_permutation", "maxe_permute_gather", "maxe_permute_scatter",
    "maxe_permute_csr", "maxe_handle_csr", "maxe_handle_tuning", "maxe_nnz_entropy", "maxe_spmv", "maxe_spmv_host", "maxe_spmm", "maxe_power_iteration",
    "maxe_handle_destroy", "maxe_device_status", "maxe_status_str", "maxe_version",
    "maxe_batch_create", "maxe_batch_set", "maxe_batch_run", "maxe_batch_destroy", "maxe_batch_tune",
    "maxe_batch_plan_info", "maxe_vec_norm_gather", "maxe_vec_dot_gather", "maxe_entropy_levels",
    "maxe_nnz_histogram", "maxe_gradient_permutation", "maxe_coo_spmv", "maxe_handle_coo",
    "maxe_power_iteration_history", "maxe_set_wait_limit_ns", "maxe_selftest_wait", "maxe_batch_plan_shape",
]
MAXE_BATCH_SCATTER_Y = 0x1


class MaxeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)}")
        self.status = status


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)),
                ("ctx", ctypes.c_void_p)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("k", ctypes.c_int32), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64),
                ("Y", ctypes.c_void_p), ("ldy", ctypes.c_int64), ("flags", ctypes.c_uint32)]


class _Csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("dtype", ctypes.c_int)]


_lock = threading.Lock()
_lib = None
_live: dict[int, torch.Tensor] = {}  # allocations handed to the library


def _torch_alloc(nbytes, ctx, stream):
    try:
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
    except Exception:  # out of memory -> NULL -> MAXE_ERR_OOM
        return None
    p = t.data_ptr()
    _live[p] = t
    return p


def _torch_free(ptr, ctx, stream):
    if ptr:
        _live.pop(int(ptr), None)


_ALLOC = _Allocator(_Allocator._fields_[0][1](_torch_alloc), _Allocator._fields_[1][1](_torch_free), None)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libmaxe.so; raises if it has not been built (no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libmaxe.so not built ({_build.LIB}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        st = ctypes.c_int
        sig = {
            "maxe_build_permutation": [ctypes.c_uint64, I32, I32, P, P, P],
            "maxe_invert_permutation": [P, I32, P, P],
            "maxe_permute_gather": [P, I32, I32, P, P, P],
            "maxe_permute_scatter": [P, I32, I32, P, P, P],
            "maxe_permute_csr": [ctypes.POINTER(_Csr), P, P, U32, P, P, ctypes.POINTER(P)],
            "maxe_handle_csr": [P, ctypes.POINTER(_Csr), ctypes.POINTER(P), ctypes.POINTER(P)],
            "maxe_handle_tuning": [P, ctypes.POINTER(I32)],
            "maxe_nnz_entropy": [P, I32, I32, ctypes.c_double, ctypes.POINTER(ctypes.c_double), P, P, P],
            "maxe_spmv": [P, P, P, U32, P],
            "maxe_spmv_host": [P, P, P, P, P, U32, P],
            "maxe_spmm": [P, I32, P, I64, P, I64, U32, P],
            "maxe_power_iteration": [P, P, I32, P, ctypes.POINTER(ctypes.c_double), P],
            "maxe_power_iteration_history": [P, P, I32, P, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), P],
            "maxe_handle_destroy": [P],
            "maxe_device_status": [P],
            "maxe_set_wait_limit_ns": [ctypes.c_uint64],
            "maxe_selftest_wait": [P],
            "maxe_batch_create": [I32, P, P, ctypes.POINTER(P)],
            "maxe_batch_set": [P, ctypes.POINTER(_BatchItem), I32],
            "maxe_batch_run": [P, P],
            "maxe_batch_destroy": [P],
            "maxe_batch_tune": [P, I32, P],
            "maxe_batch_plan_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32)],
            "maxe_batch_plan_shape": [P, ctypes.POINTER(I32)],
            "maxe_vec_norm_gather": [P, I32, I32, P, P, P, P],
            "maxe_entropy_levels": [P, I32, I32, I32, ctypes.c_double, P, P],
            "maxe_nnz_histogram": [P, I32, P, P],
            "maxe_coo_spmv": [P, P, P, ctypes.c_uint32, P],
            "maxe_handle_coo": [P, ctypes.POINTER(ctypes.c_void_p)],
            "maxe_gradient_permutation": [P, I32, ctypes.c_uint64, I32, P, P, P, P],
            "maxe_vec_dot_gather": [P, I32, I32, P, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = st
        lib.maxe_status_str.argtypes = [ctypes.c_int]
        lib.maxe_status_str.restype = ctypes.c_char_p
        lib.maxe_version.argtypes = []
        lib.maxe_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def status_str(s: int) -> str:
    try:
        return load().maxe_status_str(s).decode()
    except Exception:
        return f"status {s}"


def _check(s: int, what: str):
    if s != MAXE_OK:
        raise MaxeError(s, what)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


def _view(ptr: int | None, n: int, dtype: torch.dtype) -> torch.Tensor | None:
    if not ptr:
        return None
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    if dtype == torch.bfloat16:
        return torch.as_tensor(_DevArray(ptr, n, "<i2"), device="cuda").view(torch.bfloat16)
    ts = {torch.int32: "<i4", torch.float32: "<f4", torch.float64: "<f8"}[dtype]
    return torch.as_tensor(_DevArray(ptr, n, ts), device="cuda")


class Handle:
    """Library-owned permuted matrix A' = P_r A P_c (opaque maxe_handle*)."""

    def __init__(self, ptr: int, rows: int, cols: int, nnz: int, dtype: int, keep):
        self.ptr = ptr
        self.rows, self.cols, self.nnz, self.dtype = rows, cols, nnz, dtype
        self._keep = keep

    @property
    def vec_dtype(self) -> torch.dtype:
        return VEC_TORCH[self.dtype]

    def csr(self):
        """(rowptr, col, val, rperm, cperm) as zero-copy torch views of the handle's arrays."""
        v = _Csr()
        rp, cp = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().maxe_handle_csr(ctypes.c_void_p(self.ptr), ctypes.byref(v), ctypes.byref(rp), ctypes.byref(cp)),
               "maxe_handle_csr")
        return (_view(v.rowptr, self.rows + 1, torch.int32), _view(v.col, self.nnz, torch.int32),
                _view(v.val, self.nnz, VAL_TORCH[self.dtype]), _view(rp.value, self.rows, torch.int32),
                _view(cp.value, self.cols, torch.int32))

    def coo_rows(self):
        """COO row index of every entry (zero-copy view), for handles made with coo=True."""
        r = ctypes.c_void_p()
        _check(load().maxe_handle_coo(ctypes.c_void_p(self.ptr), ctypes.byref(r)), "maxe_handle_coo")
        return _view(r.value, self.nnz, torch.int32)

    def items_per_lane(self) -> int:
        """Entries per lane of the SpMV kernel variant this handle uses (8 or 16)."""
        return self._tuning() & 0xFF

    def xslice(self) -> bool:
        """True when SpMV runs on the x-sliced form (MAXE_XSLICE, kept by the autotuner or forced)."""
        return bool(self._tuning() & 0x200)

    def xslice_prefetch(self) -> bool:
        """True when the x-sliced SpMV runs its L2 prefetch cursor (large cells)."""
        return bool(self._tuning() & 0x400)

    def xslice_pairs(self) -> bool:
        """True when the x-sliced SpMV runs each tile on a cluster of two CTAs (column halves)."""
        return bool(self._tuning() & 0x800)

    def spmm_rows(self) -> bool:
        """True when SpMM takes one row per group of lanes (MAXE_SPMM_ROWS, or kept by the autotuner)."""
        return bool(self._tuning() & 0x1000)

    def spmm_rows_prefetch(self) -> bool:
        """True when the rows SpMM kernel prefetches each lane group's next X rows (autotuned)."""
        return bool(self._tuning() & 0x40000)

    def xslice_ahead(self) -> int:
        """L2 prefetch distance (entries) of the x-sliced SpMV's entry stream (0: none)."""
        return 512 * ((self._tuning() >> 15) & 7)

    def batch_spmm_kernel(self) -> str:
        """SpMM kernel of the handle's batch plan: "passes", "lanes" or "rows"."""
        return ("passes", "lanes", "rows", "passes")[(self._tuning() >> 13) & 3]

    def spmm_lanes(self) -> bool:
        """True when SpMM spreads the k columns across lanes (else column passes)."""
        return bool(self._tuning() & 0x100)

    def _tuning(self) -> int:
        v = ctypes.c_int32()
        _check(load().maxe_handle_tuning(ctypes.c_void_p(self.ptr), ctypes.byref(v)), "maxe_handle_tuning")
        return v.value

    def close(self):
        if self.ptr:
            load().maxe_handle_destroy(ctypes.c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ entry points

def maxe_build_permutation(seed: int, n: int, tag: int, perm: torch.Tensor | None = None, stream=None):
    """perm[new] = old, sorted by key(seed, tag, i) (Section 3)."""
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _dev(perm, torch.int32, "perm")
    _check(load().maxe_build_permutation(ctypes.c_uint64(seed & (2**64 - 1)), n, tag, _ptr(perm),
                                         ctypes.byref(_ALLOC), ctypes.c_void_p(_stream(stream))),
           "maxe_build_permutation")
    return perm


def maxe_invert_permutation(perm: torch.Tensor, stream=None):
    _dev(perm, torch.int32, "perm")
    inv = torch.empty_like(perm)
    _check(load().maxe_invert_permutation(_ptr(perm), perm.numel(), _ptr(inv), ctypes.c_void_p(_stream(stream))),
           "maxe_invert_permutation")
    return inv


def maxe_permute_gather(perm: torch.Tensor, x: torch.Tensor, stream=None):
    """out[i] = x[perm[i]]  (x' = P_c^{-1} x)."""
    _dev(perm, torch.int32, "perm")
    out = torch.empty(perm.numel(), dtype=x.dtype, device="cuda")
    _check(load().maxe_permute_gather(_ptr(perm), perm.numel(), x.element_size(), _ptr(x), _ptr(out),
                                      ctypes.c_void_p(_stream(stream))), "maxe_permute_gather")
    return out


def maxe_permute_scatter(perm: torch.Tensor, y: torch.Tensor, stream=None):
    """out[perm[i]] = y[i]  (y = P_r^{-1} y')."""
    _dev(perm, torch.int32, "perm")
    out = torch.empty(perm.numel(), dtype=y.dtype, device="cuda")
    _check(load().maxe_permute_scatter(_ptr(perm), perm.numel(), y.element_size(), _ptr(y), _ptr(out),
                                       ctypes.c_void_p(_stream(stream))), "maxe_permute_scatter")
    return out


def maxe_permute_csr(rows: int, cols: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                     rperm: torch.Tensor | None = None, cperm: torch.Tensor | None = None, validate: bool = False,
                     stream=None, autotune: bool = False, items16: bool = False, spmm_lanes: bool = False,
                     equal_rows: bool = False, coo: bool = False, xslice: bool = False,
                     xs_pairs: bool | None = None, spmm_rows: bool = False, spmm_rows_pf: bool = False) -> Handle:
    """Handle of A' = P_r A P_c (Eq. 1) with ascending columns; None perms = identity.
    xs_pairs: None lets the library decide whether the x-sliced form runs its
    tiles on CTA pairs (column halves); True / False forces it on / off."""
    code = {torch.float64: MAXE_F64, torch.float32: MAXE_F32, torch.bfloat16: MAXE_BF16}[val.dtype]
    _dev(rowptr, torch.int32, "rowptr")
    _dev(col, torch.int32, "col")
    _dev(val, val.dtype, "val")
    if rperm is not None:
        _dev(rperm, torch.int32, "rperm")
    if cperm is not None:
        _dev(cperm, torch.int32, "cperm")
    A = _Csr(rows, cols, col.numel(), rowptr.data_ptr(), col.data_ptr() if col.numel() else None,
             val.data_ptr() if val.numel() else None, code)
    out = ctypes.c_void_p()
    flags = ((MAXE_VALIDATE if validate else 0) | (MAXE_AUTOTUNE if autotune else 0) | (MAXE_ITEMS16 if items16 else 0)
             | (MAXE_SPMM_LANES if spmm_lanes else 0) | (MAXE_EQUAL_ROWS if equal_rows else 0)
             | (MAXE_COO if coo else 0) | (MAXE_XSLICE if xslice else 0)
             | (0 if xs_pairs is None else (MAXE_XS_PAIRS if xs_pairs else MAXE_XS_SINGLE))
             | (MAXE_SPMM_ROWS if spmm_rows else 0) | (MAXE_SPMM_ROWS_PF if spmm_rows_pf else 0))
    _check(load().maxe_permute_csr(ctypes.byref(A), _ptr(rperm), _ptr(cperm), flags,
                                   ctypes.byref(_ALLOC), ctypes.c_void_p(_stream(stream)), ctypes.byref(out)),
           "maxe_permute_csr")
    return Handle(out.value, rows, cols, col.numel(), code, keep=None)


def maxe_nnz_entropy(h: Handle, gr: int, gc: int, base: float = 2.0, counts: bool = True, stream=None):
    """(H, counts[gr, gc] int64 or None) of the nonzero block-grid histogram (Section 4)."""
    H = ctypes.c_double()
    cnt = torch.empty(gr * gc, dtype=torch.int64, device="cuda") if counts else None
    _check(load().maxe_nnz_entropy(ctypes.c_void_p(h.ptr), gr, gc, float(base), ctypes.byref(H), _ptr(cnt),
                                   ctypes.byref(_ALLOC), ctypes.c_void_p(_stream(stream))), "maxe_nnz_entropy")
    return H.value, (cnt.view(gr, gc) if counts else None)


def maxe_spmv(h: Handle, x: torch.Tensor, y: torch.Tensor | None = None, permuted: bool = False, stream=None):
    """y = A x (original space), or y' = A' x' with permuted=True (MAXE_VEC_PERMUTED)."""
    _dev(x, h.vec_dtype, "x")
    if x.numel() != h.cols:
        raise ValueError("x has the wrong length")
    if y is None:
        y = torch.empty(h.rows, dtype=h.vec_dtype, device="cuda")
    _dev(y, h.vec_dtype, "y")
    _check(load().maxe_spmv(ctypes.c_void_p(h.ptr), _ptr(x), _ptr(y), MAXE_VEC_PERMUTED if permuted else 0,
                            ctypes.c_void_p(_stream(stream))), "maxe_spmv")
    return y


def _host(t: torch.Tensor, dtype, n: int, name: str) -> torch.Tensor:
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t


def maxe_spmv_host(h: Handle, x_host: torch.Tensor, y_host: torch.Tensor, x_dev: torch.Tensor, y_dev: torch.Tensor,
                   permuted: bool = False, stream=None):
    """y = A x from host memory in one library call: x_host is copied into the
    device scratch x_dev, the product written to y_dev and copied into y_host,
    all enqueued on `stream`; y_host holds y once the stream has passed the
    call.  Pinned host tensors let the copies run asynchronously."""
    _host(x_host, h.vec_dtype, h.cols, "x_host")
    _host(y_host, h.vec_dtype, h.rows, "y_host")
    _dev(x_dev, h.vec_dtype, "x_dev")
    _dev(y_dev, h.vec_dtype, "y_dev")
    if x_dev.numel() != h.cols or y_dev.numel() != h.rows:
        raise ValueError("x_dev / y_dev have the wrong length")
    _check(load().maxe_spmv_host(ctypes.c_void_p(h.ptr), _ptr(x_host), _ptr(y_host), _ptr(x_dev), _ptr(y_dev),
                                 MAXE_VEC_PERMUTED if permuted else 0, ctypes.c_void_p(_stream(stream))),
           "maxe_spmv_host")
    return y_host


def maxe_coo_spmv(h: Handle, x: torch.Tensor, y: torch.Tensor | None = None, permuted: bool = False, stream=None):
    """y = A x over the handle's COO triplets (Section 2); needs a handle made with coo=True."""
    _dev(x, h.vec_dtype, "x")
    if x.numel() != h.cols:
        raise ValueError("x has the wrong length")
    if y is None:
        y = torch.empty(h.rows, dtype=h.vec_dtype, device="cuda")
    _dev(y, h.vec_dtype, "y")
    _check(load().maxe_coo_spmv(ctypes.c_void_p(h.ptr), _ptr(x), _ptr(y), MAXE_VEC_PERMUTED if permuted else 0,
                                ctypes.c_void_p(_stream(stream))), "maxe_coo_spmv")
    return y


def maxe_spmm(h: Handle, X: torch.Tensor, Y: torch.Tensor | None = None, permuted: bool = False, stream=None):
    """Y = A X for row-major X (cols x k); permuted=True keeps both in the permuted space."""
    if X.dim() != 2 or X.shape[0] != h.cols or X.stride(1) != 1:
        raise ValueError("X must be (cols, k) with unit column stride")
    if X.dtype != h.vec_dtype or not X.is_cuda:
        raise TypeError("X has the wrong dtype/device")
    k = X.shape[1]
    if Y is None:
        Y = torch.empty(h.rows, k, dtype=h.vec_dtype, device="cuda")
    if Y.stride(1) != 1 or Y.shape != (h.rows, k):
        raise ValueError("Y must be (rows, k) with unit column stride")
    _check(load().maxe_spmm(ctypes.c_void_p(h.ptr), k, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                            MAXE_VEC_PERMUTED if permuted else 0, ctypes.c_void_p(_stream(stream))), "maxe_spmm")
    return Y


def maxe_power_iteration(h: Handle, v0: torch.Tensor, steps: int, stream=None, history: bool = False):
    """(lambda, v) after `steps` normalised products in the original space; with
    history, (lambda, v, Rayleigh quotient after every step as a numpy array)."""
    _dev(v0, h.vec_dtype, "v0")
    v = torch.empty_like(v0)
    lam = ctypes.c_double()
    if history:
        hist = (ctypes.c_double * max(steps, 1))()
        _check(load().maxe_power_iteration_history(ctypes.c_void_p(h.ptr), _ptr(v0), steps, _ptr(v),
                                                   ctypes.byref(lam), hist, ctypes.c_void_p(_stream(stream))),
               "maxe_power_iteration_history")
        return lam.value, v, np.array(hist[:steps], dtype=np.float64)
    _check(load().maxe_power_iteration(ctypes.c_void_p(h.ptr), _ptr(v0), steps, _ptr(v), ctypes.byref(lam),
                                       ctypes.c_void_p(_stream(stream))), "maxe_power_iteration")
    return lam.value, v


def maxe_device_status(stream=None) -> int:
    return load().maxe_device_status(ctypes.c_void_p(_stream(stream)))


def maxe_set_wait_limit_ns(ns: int):
    """Bounded device waits give up after `ns` (0: the 2 s default)."""
    _check(load().maxe_set_wait_limit_ns(ctypes.c_uint64(int(ns))), "maxe_set_wait_limit_ns")


def maxe_selftest_wait(stream=None):
    """Launch a wait on a flag nothing sets; it runs out after the wait limit."""
    _check(load().maxe_selftest_wait(ctypes.c_void_p(_stream(stream))), "maxe_selftest_wait")


def maxe_version() -> str:
    return load().maxe_version().decode()


def from_csr(A, rperm=None, cperm=None, validate=False, stream=None, autotune=False, items16=False,
             spmm_lanes=False, equal_rows=False, coo=False, xslice=False, xs_pairs=None, spmm_rows=False,
             spmm_rows_pf=False) -> Handle:
    """Handle from a workloads.CSR already on the GPU."""
    return maxe_permute_csr(A.rows, A.cols, A.rowptr, A.col, A.val, rperm, cperm, validate, stream, autotune, items16,
                            spmm_lanes, equal_rows, coo, xslice, xs_pairs, spmm_rows, spmm_rows_pf)


class Batch:
    """Batched persistent SpMV/SpMM over many handles (maxe_batch_*).

    items: list of (handle, X, Y, scatter_y) with X (cols x k) in the permuted
    space and Y (rows x k) written in the permuted space, or through rperm when
    scatter_y is True.  Tensors must stay alive while the batch may run."""

    def __init__(self, capacity: int, stream=None):
        out = ctypes.c_void_p()
        _check(load().maxe_batch_create(capacity, ctypes.byref(_ALLOC), ctypes.c_void_p(_stream(stream)),
                                        ctypes.byref(out)), "maxe_batch_create")
        self.ptr = out.value
        self._keep = []

    def set(self, items):
        arr = (_BatchItem * max(len(items), 1))()
        keep = []
        for i, (h, X, Y, scatter) in enumerate(items):
            if X.dim() == 1:
                X = X.view(-1, 1)
            if Y.dim() == 1:
                Y = Y.view(-1, 1)
            k = X.shape[1]
            if X.dtype != h.vec_dtype or Y.dtype != h.vec_dtype or Y.shape[1] != k:
                raise TypeError("batch item vectors do not match the handle")
            arr[i] = _BatchItem(h.ptr, k, X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
                                MAXE_BATCH_SCATTER_Y if scatter else 0)
            keep += [h, X, Y]
        _check(load().maxe_batch_set(ctypes.c_void_p(self.ptr), arr, len(items)), "maxe_batch_set")
        self._keep = keep

    def run(self, stream=None):
        _check(load().maxe_batch_run(ctypes.c_void_p(self.ptr), ctypes.c_void_p(_stream(stream))), "maxe_batch_run")

    def close(self):
        if self.ptr:
            load().maxe_batch_destroy(ctypes.c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def maxe_batch_tune(h: Handle, k: int, stream=None):
    _check(load().maxe_batch_tune(ctypes.c_void_p(h.ptr), k, ctypes.c_void_p(_stream(stream))), "maxe_batch_tune")


def maxe_batch_plan_info(h: Handle):
    """(entries per warp task, tasks, entries per lane) of the handle's batch plan."""
    H, t, it = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().maxe_batch_plan_info(ctypes.c_void_p(h.ptr), ctypes.byref(H), ctypes.byref(t), ctypes.byref(it)),
           "maxe_batch_plan_info")
    return H.value, t.value, it.value


def maxe_batch_plan_shape(h: Handle) -> int:
    """CTAs per SM the handle's batch plan asks of a launch (0: as many as fit)."""
    v = ctypes.c_int32()
    _check(load().maxe_batch_plan_shape(ctypes.c_void_p(h.ptr), ctypes.byref(v)), "maxe_batch_plan_shape")
    return v.value


def maxe_vec_norm_gather(Q: torch.Tensor | None, w: torch.Tensor, u: torch.Tensor, scratch: torch.Tensor, stream=None):
    """u[j] = w[Q[j]] / ||w||_2 (FP64 norm); scratch: >= 514 float64 on the device."""
    _check(load().maxe_vec_norm_gather(_ptr(Q), w.numel(), w.element_size(), _ptr(w), _ptr(u), _ptr(scratch),
                                       ctypes.c_void_p(_stream(stream))), "maxe_vec_norm_gather")


def maxe_vec_dot_gather(Q: torch.Tensor | None, u: torch.Tensor, w: torch.Tensor, scratch: torch.Tensor,
                        out: torch.Tensor, stream=None):
    """out[0] = sum_j u[j] * w[Q[j]] (FP64)."""
    _check(load().maxe_vec_dot_gather(_ptr(Q), u.numel(), u.element_size(), _ptr(u), _ptr(w), _ptr(scratch),
                                      _ptr(out), ctypes.c_void_p(_stream(stream))), "maxe_vec_dot_gather")


def maxe_entropy_levels(counts: torch.Tensor, L: int, base: float = 2.0, stream=None) -> torch.Tensor:
    """(L, L) block entropies of a (gr, gc) int64 count grid (Section 5, hierarchical 2-D entropy)."""
    _dev(counts, torch.int64, "counts")
    gr, gc = counts.shape
    out = torch.empty(L * L, dtype=torch.float64, device="cuda")
    _check(load().maxe_entropy_levels(_ptr(counts), gr, gc, L, float(base), _ptr(out),
                                      ctypes.c_void_p(_stream(stream))), "maxe_entropy_levels")
    return out.view(L, L)


def _csr_struct(A) -> _Csr:
    code = {torch.float64: MAXE_F64, torch.float32: MAXE_F32, torch.bfloat16: MAXE_BF16}[A.val.dtype]
    return _Csr(A.rows, A.cols, A.col.numel(), A.rowptr.data_ptr(),
                   A.col.data_ptr() if A.col.numel() else None, A.val.data_ptr() if A.val.numel() else None, code)


def maxe_nnz_histogram(A, axis: int, stream=None) -> torch.Tensor:
    """Entries per row (axis 0) or per column (axis 1) of a CSR on the GPU (Section 5, appendix)."""
    _dev(A.rowptr, torch.int32, "rowptr")
    hist = torch.empty(A.rows if axis == 0 else A.cols, dtype=torch.int32, device="cuda")
    s = _csr_struct(A)
    _check(load().maxe_nnz_histogram(ctypes.byref(s), int(axis), _ptr(hist), ctypes.c_void_p(_stream(stream))),
           "maxe_nnz_histogram")
    return hist


def maxe_gradient_permutation(hist: torch.Tensor, seed: int, tag: int, stream=None):
    """(perm, pivot): cut at the steepest histogram step, riffle, random order in each
    half of the shuffled deck (appendix, gradient-based permutations). pivot is a
    one-element device tensor."""
    _dev(hist, torch.int32, "hist")
    n = hist.numel()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    pivot = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(load().maxe_gradient_permutation(_ptr(hist), n, ctypes.c_uint64(seed & (2**64 - 1)), tag, _ptr(perm),
                                            _ptr(pivot), ctypes.byref(_ALLOC), ctypes.c_void_p(_stream(stream))),
           "maxe_gradient_permutation")
    return perm, pivot


def gradient_perms(A, seed: int, columns: bool = False, stream=None):
    """(rperm, cperm) of the gradient-based row (G-R) or row+column (G-C) permutation."""
    rperm, _ = maxe_gradient_permutation(maxe_nnz_histogram(A, 0, stream), seed, 0, stream)
    cperm = None
    if columns:
        cperm, _ = maxe_gradient_permutation(maxe_nnz_histogram(A, 1, stream), seed, 1, stream)
    return rperm, cperm
