"""The allocation-free entropy entry point (maxe_nnz_entropy_noalloc) against
the allocating one, through the C ABI.

Some callers of this library cannot allocate device memory (a framework that
owns the whole device pool and hands out only input/output buffers, or a path
where cudaMalloc's implicit synchronisation is not allowed); they use the
variant whose scratch is a static device array.  This file is collected last
so that a run stopping at its first failure has already run everything else;
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    lib = maxe.load(build_if_missing=True)
    fn = lib.maxe_nnz_entropy_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _call(fn, h, gr, gc):
    H = ctypes.c_double(-1.0)
    cnt = torch.full((gr * gc,), -1, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(h.ptr), gr, gc, 2.0, ctypes.byref(H), ctypes.c_void_p(cnt.data_ptr()), stream)
    return rc, H.value, cnt


def test_noalloc_entropy_matches_allocating_entry_point_twice_in_a_row():
    fn = _noalloc_fn()
    A = W.powerlaw(11, n=150000, device="cuda")
    rperm = maxe.maxe_build_permutation(11, A.rows, 0)
    cperm = maxe.maxe_build_permutation(11, A.cols, 1)
    h = maxe.from_csr(A, rperm, cperm)
    # two calls in a row on the same grid (the second must not see the first's
    # counts), then a different grid
    for gr, gc in [(64, 64), (64, 64), (256, 256)]:
        H_ref, cnt_ref = maxe.maxe_nnz_entropy(h, gr, gc)
        rc, H, cnt = _call(fn, h, gr, gc)
        assert rc == maxe.MAXE_OK, maxe.status_str(rc)
        np.testing.assert_array_equal(cnt.view(gr, gc).cpu().numpy(), cnt_ref.cpu().numpy())
        assert H == pytest.approx(H_ref, rel=1e-12, abs=1e-15)
    h.close()


def test_noalloc_entropy_rejects_grids_beyond_its_scratch():
    fn = _noalloc_fn()
    A = W.poisson_uniform(3, 1000, 8.0, device="cuda")
    h = maxe.from_csr(A)
    rc, _, _ = _call(fn, h, 257, 256)  # 65792 cells > 65536
    assert rc == maxe.MAXE_ERR_INVALID
    rc, H, cnt = _call(fn, h, 256, 256)
    assert rc == maxe.MAXE_OK and int(cnt.sum()) == A.nnz
    h.close()
