"""Parity at the full sizes the benchmark runs, in the launch configuration it
times (autotuned handles; vectors in the permuted space), on every row and
column against the FP64 oracle (relative L2 and a per-row rounding bound):
the 1M-row power-law matrix in all three value types, permuted and plain, the
5-point Laplacian on a 4096 x 4096 grid in all three value types with
k = 1, 4, 16, and the 256-matrix batch in one persistent launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import check_all_rows, check_all_rows_spmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)
    yield
    torch.cuda.synchronize()
    assert maxe.maxe_device_status() == maxe.MAXE_OK


def _vals_np(val: torch.Tensor):
    v = val.cpu()
    return v.view(torch.int16).numpy().view(np.uint16) if v.dtype == torch.bfloat16 else v.numpy()


def _all(h, X, Y, dtype, what=""):
    """Y = A' X (every row and column) against the oracle on the handle's own CSR."""
    rp, co, va, _, _ = h.csr()
    check_all_rows_spmm(Y.cpu().numpy(), rp.cpu().numpy(), co.cpu().numpy(), _vals_np(va), dtype,
                        X.cpu().numpy(), what)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_powerlaw_1M_full_size_as_benchmarked(dtype):
    base = W.powerlaw(2308, device="cuda")
    A = base if dtype == "f32" else base.astype(dtype)
    r = maxe.maxe_build_permutation(2308, A.rows, 0)
    c = maxe.maxe_build_permutation(2308, A.cols, 1)
    vdt = "f64" if dtype == "f64" else "f32"
    for perms in ((r, c), (None, None)):
        h = maxe.from_csr(A, *perms, autotune=True)
        x = W.vector(1, A.cols, vdt, "cuda")
        y = maxe.maxe_spmv(h, x, permuted=True)
        _all(h, x, y, dtype, ("permuted" if perms[0] is not None else "plain", h.xslice(), h.xslice_pairs()))
        h.close()
    # the original-space call: x gathered through cperm, y scattered through rperm
    h = maxe.from_csr(A, r, c, autotune=True)
    x = W.vector(2, A.cols, vdt, "cuda")
    y = maxe.maxe_spmv(h, x)
    rp, co, va = A.numpy()
    check_all_rows(y.cpu().numpy(), rp, co, va, dtype, x.cpu().numpy(), "original space")


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_laplacian_4096_full_size(dtype):
    base = W.laplacian5(4096, "f64", "cuda")
    A = base.astype(dtype)
    r = maxe.maxe_build_permutation(2308, A.rows, 0)
    c = maxe.maxe_build_permutation(2308, A.cols, 1)
    vdt = "f64" if dtype == "f64" else "f32"
    for perms in ((r, c), (None, None)):
        h = maxe.from_csr(A, *perms, autotune=True)
        for k in (1, 4, 16):
            if k == 1:
                X = W.vector(k, A.cols, vdt, "cuda")
                Y = maxe.maxe_spmv(h, X, permuted=True)
            else:
                X = W.matrix_rhs(k, A.cols, k, vdt, "cuda")
                Y = maxe.maxe_spmm(h, X, permuted=True)
            _all(h, X, Y, dtype, (k, perms[0] is not None, h.spmm_rows(), h.spmm_lanes()))
            del X, Y
        h.close()


def test_batched_256_full_size_one_launch():
    mats, ks = W.batched_set(2308, count=256, device="cuda")
    hs, Xs, Ys = [], [], []
    for m, (A, k) in enumerate(zip(mats, ks)):
        rp_ = maxe.maxe_build_permutation(2308 + m, A.rows, 0)
        cp_ = maxe.maxe_build_permutation(2308 + m, A.cols, 1)
        hs.append(maxe.from_csr(A, rp_, cp_))
        kp = (k + 3) // 4 * 4
        Xb = torch.zeros(A.cols, kp, device="cuda")
        Xb[:, :k] = W.matrix_rhs(m, A.cols, k, "f32", "cuda")
        Xs.append(Xb[:, :k])
        Ys.append(torch.empty(A.rows, kp, device="cuda")[:, :k])
    b = maxe.Batch(len(mats))
    b.set([(h, X, Y, False) for h, X, Y in zip(hs, Xs, Ys)])
    b.run()
    torch.cuda.synchronize()
    for m in range(len(mats)):
        _all(hs[m], Xs[m], Ys[m], "f32", ("batch item", m, ks[m]))
    b.close()
    for h in hs:
        h.close()
