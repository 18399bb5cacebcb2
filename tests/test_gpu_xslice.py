"""GPU parity of the x-sliced SpMV (x staged in shared memory by column slices,
rows owned by warps, tiles on one CTA or on a cluster of two CTAs that split
the columns): every row within the FP tolerance of the FP64 oracle in both
spaces, deterministic, with more tiles than SMs, and the CSR kernel taking over
for unaligned x."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import EDGE_KINDS, TOL, check_all_rows, code, edge_matrix, oracle_permuted, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)


def _perms(A, seed):
    return maxe.maxe_build_permutation(seed, A.rows, 0), maxe.maxe_build_permutation(seed, A.cols, 1)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("kind", EDGE_KINDS + ["mixed"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_xslice_spmv_against_oracle(kind, dtype, pairs):
    if kind == "mixed":
        L = np.random.default_rng(7).choice([0, 1, 7, 8, 9, 255, 256, 257, 900], 3000)
        A = W.from_lengths(7, L, 40000, dtype)
    else:
        A = edge_matrix(kind, dtype, seed=8)
    rperm, cperm = _perms(A, 31)
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, xslice=True, xs_pairs=pairs)
    assert h.xslice() == (A.nnz > 0)
    assert h.xslice_pairs() == (A.nnz > 0 and pairs and dtype != "f64")  # FP64 values never run pairs
    vd = "f64" if dtype == "f64" else "f32"
    x = W.vector(9, A.cols, vd, "cuda")
    rp, co, va = A.numpy()
    y = torch.full((A.rows,), float("nan"), dtype=x.dtype, device="cuda")
    maxe.maxe_spmv(h, x, y)  # original space: x gathered, y scattered through rperm
    assert not torch.isnan(y).any()
    check_all_rows(y.cpu().numpy(), rp, co, va, dtype, x.cpu().numpy(), "original space")
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    xp = x[cperm.long()].contiguous()
    yp = maxe.maxe_spmv(h, xp, permuted=True)
    check_all_rows(yp.cpu().numpy(), nrp, nco, nva, dtype, xp.cpu().numpy(), "permuted space")
    assert torch.equal(maxe.maxe_spmv(h, xp, permuted=True), yp)  # deterministic


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_xslice_many_tiles_per_cta(dtype):
    """More row tiles than SMs (the 5-point Laplacian, 2.9M rows: the tiles are
    bounded by the accumulators that fit in shared memory), so the CTAs run in
    several waves; natural order keeps the cells large (the prefetch cursor)."""
    A = W.laplacian5(1700, dtype, "cuda")
    h = maxe.from_csr(A, xslice=True)
    assert h.xslice() and h.xslice_prefetch() and not h.xslice_pairs()  # banded: uneven column halves
    x = W.vector(3, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
    y = maxe.maxe_spmv(h, x)
    rp, co, va = A.numpy()
    check_all_rows(y.cpu().numpy(), rp, co, va, dtype, x.cpu().numpy())
    ones = maxe.maxe_spmv(h, torch.ones(A.cols, dtype=x.dtype, device="cuda")).cpu().numpy().reshape(1700, 1700)
    ref1 = np.zeros((1700, 1700))
    ref1[0, :] += 1
    ref1[-1, :] += 1
    ref1[:, 0] += 1
    ref1[:, -1] += 1
    np.testing.assert_array_equal(ones, ref1)


@pytest.mark.parametrize("pairs", [None, False])
def test_xslice_powerlaw_deterministic_and_matches_csr(pairs):
    A = W.powerlaw(5, n=400000, device="cuda")
    rperm, cperm = _perms(A, 5)
    h = maxe.from_csr(A, rperm, cperm, xslice=True, xs_pairs=pairs)
    hc = maxe.from_csr(A, rperm, cperm)
    assert h.xslice() and not hc.xslice()
    assert h.xslice_pairs() == (pairs is None)  # permuted: the column halves of every tile are even
    assert not h.xslice_prefetch()  # permuted: small cells, no prefetch cursor
    x = W.vector(4, A.cols, "f32", "cuda")
    y1 = maxe.maxe_spmv(h, x)
    assert torch.equal(maxe.maxe_spmv(h, x), y1)
    assert rel_l2(y1.cpu().numpy(), maxe.maxe_spmv(hc, x).cpu().numpy()) <= 1e-6
    rp, co, va = A.numpy()
    check_all_rows(y1.cpu().numpy(), rp, co, va, "f32", x.cpu().numpy())
    # x not 16-byte aligned: the CSR kernel runs instead, same result within FP32 rounding
    xb = torch.empty(A.cols + 1, device="cuda")
    xb[1:] = x[cperm.long()]
    yu = maxe.maxe_spmv(h, xb[1:], permuted=True)
    ya = maxe.maxe_spmv(h, x[cperm.long()].contiguous(), permuted=True)
    assert rel_l2(yu.cpu().numpy(), ya.cpu().numpy()) <= 1e-6
    # the power iteration runs its products through the same kernel
    v0 = W.vector(8, A.rows, "f32", "cuda")
    lam_x, _ = maxe.maxe_power_iteration(h, v0, 5)
    lam_c, _ = maxe.maxe_power_iteration(hc, v0, 5)
    assert abs(lam_x - lam_c) <= 1e-4 * abs(lam_c)


def test_xslice_autotune_keeps_the_faster_kernel():
    A = W.powerlaw(6, n=300000, device="cuda")
    h = maxe.from_csr(A, *_perms(A, 6), autotune=True)
    x = W.vector(5, A.cols, "f32", "cuda")
    rp, co, va = A.numpy()
    y = maxe.maxe_spmv(h, x)
    check_all_rows(y.cpu().numpy(), rp, co, va, "f32", x.cpu().numpy())


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("permuted", [False, True])
def test_xslice_infinite_x_reaches_only_its_rows(dtype, permuted, pairs):
    """Lanes without an entry in a step compute nothing: infinities in x reach
    only the rows that have entries in those columns.  The infinities sit on the
    first column of every slice (of both slice widths) and on the last column."""
    lengths = np.random.default_rng(12).integers(0, 40, 5000)
    A = W.from_lengths(12, lengths, 40000, dtype)
    rperm, cperm = _perms(A, 13) if permuted else (None, None)
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, xslice=True, xs_pairs=pairs)
    assert h.xslice()
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    widths = [8192] if dtype == "f64" else [16384, 12288]
    bad = np.unique(np.r_[np.concatenate([np.arange(0, A.cols, w) for w in widths]), A.cols - 1])
    vd = "f64" if dtype == "f64" else "f32"
    xp = W.vector(14, A.cols, vd, "cuda")
    xp[torch.as_tensor(bad, device="cuda")] = float("inf")
    y = maxe.maxe_spmv(h, xp, permuted=True).cpu().numpy()
    row_of = np.repeat(np.arange(A.rows), np.diff(nrp))
    hit = np.zeros(A.rows, dtype=bool)
    hit[row_of[np.isin(nco, bad)]] = True
    assert hit.any() and (~hit).sum() > A.rows // 2
    assert np.isfinite(y[~hit]).all()
    x0 = xp.cpu().numpy().copy()
    x0[bad] = 0.0
    ref = oracle.spmv(A.rows, nrp, nco, nva, code(dtype), x0)
    assert rel_l2(y[~hit], ref[~hit]) <= TOL[dtype]
