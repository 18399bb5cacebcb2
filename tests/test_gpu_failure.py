"""Failure paths without a GPU fault: an allocator that fails on its n-th call
(every call of maxe_permute_csr and maxe_nnz_entropy returns MAXE_ERR_OOM, no
handle, and every block the library took is given back), and a bounded device
wait that runs out on a flag nothing sets (MAXE_ERR_TIMEOUT from
maxe_device_status, the kernel returns and the context stays usable)."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import check_all_rows, oracle_permuted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)


class FailingAllocator:
    """maxe_allocator over torch's caching allocator that returns NULL on call
    number `fail_at` (1-based; 0 never) and keeps count of live blocks."""

    def __init__(self, fail_at: int):
        self.fail_at = fail_at
        self.calls = 0
        self.live: dict[int, torch.Tensor] = {}
        self.freed_unknown = 0
        A = maxe._Allocator
        self._a = A._fields_[0][1](self._alloc)
        self._f = A._fields_[1][1](self._free)
        self.struct = A(self._a, self._f, None)

    def _alloc(self, nbytes, ctx, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, p, ctx, stream):
        if self.live.pop(p, None) is None:
            self.freed_unknown += 1


def _permute(A, rperm, cperm, flags, al):
    lib = maxe.load()
    csr = maxe._Csr(A.rows, A.cols, A.nnz, A.rowptr.data_ptr(), A.col.data_ptr(), A.val.data_ptr(),
                    maxe.DTYPE_CODE[A.dtype])
    out = ctypes.c_void_p()
    s = lib.maxe_permute_csr(ctypes.byref(csr), ctypes.c_void_p(rperm.data_ptr()), ctypes.c_void_p(cperm.data_ptr()),
                             flags, ctypes.byref(al.struct), None, ctypes.byref(out))
    torch.cuda.synchronize()
    return s, out.value


@pytest.mark.parametrize("flags", [0, maxe.MAXE_XSLICE, maxe.MAXE_XSLICE | maxe.MAXE_XS_PAIRS,
                                   maxe.MAXE_AUTOTUNE | maxe.MAXE_COO])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_allocator_failure_at_every_call_of_permute_csr(dtype, flags):
    A = W.from_lengths(21, np.random.default_rng(21).integers(0, 80, 3000), 40000, dtype).to("cuda")
    rperm = maxe.maxe_build_permutation(21, A.rows, 0)
    cperm = maxe.maxe_build_permutation(21, A.cols, 1)
    ok = FailingAllocator(0)
    s, h = _permute(A, rperm, cperm, flags, ok)
    assert s == maxe.MAXE_OK and h
    n_calls = ok.calls
    assert n_calls > 3
    maxe.load().maxe_handle_destroy(ctypes.c_void_p(h))
    torch.cuda.synchronize()
    assert not ok.live and ok.freed_unknown == 0  # the handle gave back all it took
    for k in range(1, n_calls + 1):
        al = FailingAllocator(k)
        s, h = _permute(A, rperm, cperm, flags, al)
        if s == maxe.MAXE_OK:
            # only the autotuner's optional blocks failed (its SpMM timing, the x-sliced form):
            # the handle is complete without them and still right
            assert flags & maxe.MAXE_AUTOTUNE, k
            handle = maxe.Handle(h, A.rows, A.cols, A.nnz, maxe.DTYPE_CODE[dtype], keep=None)
            x = W.vector(2, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
            y = maxe.maxe_spmv(handle, x)
            rp, co, va = A.numpy()
            check_all_rows(y.cpu().numpy(), rp, co, va, dtype, x.cpu().numpy())
            handle.close()
            torch.cuda.synchronize()
        else:
            assert s == maxe.MAXE_ERR_OOM, (k, s)
            assert not h
        assert not al.live, (k, len(al.live))  # nothing leaked
        assert al.freed_unknown == 0
    assert maxe.maxe_device_status() == maxe.MAXE_OK


def test_allocator_failure_in_entropy():
    A = W.from_lengths(22, np.random.default_rng(22).integers(0, 50, 2000), 3000, "f32").to("cuda")
    h = maxe.from_csr(A)
    lib = maxe.load()
    H = ctypes.c_double()
    ok = FailingAllocator(0)
    assert lib.maxe_nnz_entropy(ctypes.c_void_p(h.ptr), 16, 16, 2.0, ctypes.byref(H), None, ctypes.byref(ok.struct),
                                None) == maxe.MAXE_OK
    rp, co, _ = A.numpy()
    assert H.value == pytest.approx(oracle.nnz_entropy(A.rows, A.cols, rp, co, 16, 16)[0], rel=1e-12)
    assert ok.calls >= 1 and not ok.live
    for k in range(1, ok.calls + 1):
        al = FailingAllocator(k)
        assert lib.maxe_nnz_entropy(ctypes.c_void_p(h.ptr), 16, 16, 2.0, ctypes.byref(H), None,
                                    ctypes.byref(al.struct), None) == maxe.MAXE_ERR_OOM
        torch.cuda.synchronize()
        assert not al.live and al.freed_unknown == 0


def test_bounded_wait_runs_out_and_reports_timeout():
    """A wait on a flag nothing sets gives up after the wait limit (50 ms here),
    the kernel returns, maxe_device_status reports MAXE_ERR_TIMEOUT once, and the
    context goes on working: an x-sliced product afterwards is right."""
    A = W.powerlaw(23, n=50000, device="cuda")
    r = maxe.maxe_build_permutation(23, A.rows, 0)
    c = maxe.maxe_build_permutation(23, A.cols, 1)
    h = maxe.from_csr(A, r, c, xslice=True)
    assert maxe.maxe_device_status() == maxe.MAXE_OK
    with pytest.raises(maxe.MaxeError):
        maxe.maxe_set_wait_limit_ns(61 * 10**9)
    maxe.maxe_set_wait_limit_ns(50_000_000)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        maxe.maxe_selftest_wait()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert 0.04 <= dt < 10.0, dt
        assert maxe.maxe_device_status() == maxe.MAXE_ERR_TIMEOUT
        assert maxe.maxe_device_status() == maxe.MAXE_OK  # reported once, then cleared
        # products with the short limit still finish: their waits are far shorter
        x = W.vector(3, A.cols, "f32", "cuda")
        xp = x[c.long()].contiguous()
        y = maxe.maxe_spmv(h, xp, permuted=True)
        nrp, nco, nva = oracle_permuted(A.to("cpu"), r, c)
        check_all_rows(y.cpu().numpy(), nrp, nco, nva, "f32", xp.cpu().numpy())
        assert maxe.maxe_device_status() == maxe.MAXE_OK
    finally:
        maxe.maxe_set_wait_limit_ns(0)
    h.close()
