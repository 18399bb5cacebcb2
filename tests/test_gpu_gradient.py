"""GPU parity of the gradient-based permutations (Section 5; the appendix's
G-R and G-C formats): histograms and permutations bit-exact against the
oracle, products through the permuted handle within the FP tolerance."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import EDGE_KINDS, TOL, code, edge_matrix, oracle_permuted, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)


@pytest.mark.parametrize("kind", EDGE_KINDS)
def test_histograms_bit_exact(kind):
    A = edge_matrix(kind, "f32", seed=4)
    rp, co, _ = A.numpy()
    Ad = A.to("cuda")
    for axis in (0, 1):
        got = maxe.maxe_nnz_histogram(Ad, axis).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.nnz_histogram(A.rows, A.cols, rp, co, axis))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 4095, 4096, 4097, 8193, 100003, 1 << 20])
@pytest.mark.parametrize("spread", [3, 1000])
def test_gradient_permutation_bit_exact(n, spread):
    g = np.random.default_rng(n * 7 + spread)
    h = g.integers(0, spread, n).astype(np.int32)  # spread 3: ties everywhere
    for seed, tag in ((0, 0), (2308, 1), (2**64 - 1, 0)):
        perm, pivot = maxe.maxe_gradient_permutation(torch.from_numpy(h).cuda(), seed, tag)
        po, pvo = oracle.gradient_permutation(h, seed, tag)
        np.testing.assert_array_equal(perm.cpu().numpy(), po)
        assert int(pivot.item()) == pvo


@pytest.mark.parametrize("cut", [1, 17, 500000, 999999])
def test_gradient_permutation_single_step(cut):
    n = 1 << 20
    h = np.full(n, 3, dtype=np.int32)
    h[:cut] = 40
    perm, pivot = maxe.maxe_gradient_permutation(torch.from_numpy(h).cuda(), 5, 0)
    assert int(pivot.item()) == cut
    np.testing.assert_array_equal(perm.cpu().numpy(), oracle.gradient_permutation(h, 5, 0)[0])


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("columns", [False, True])
def test_gradient_shuffled_products(dtype, columns):
    """G-R / G-C permutations applied through maxe_permute_csr: CSR bit-exact,
    products within tolerance, entropy counts bit-exact."""
    A = W.clustered_heavy(3, n=30000, heavy_len=600, dtype=dtype)
    rp, co, va = A.numpy()
    Ad = A.to("cuda")
    rperm, cperm = maxe.gradient_perms(Ad, 77, columns=columns)
    ro, _ = oracle.gradient_permutation(oracle.nnz_histogram(A.rows, A.cols, rp, co, 0), 77, 0)
    np.testing.assert_array_equal(rperm.cpu().numpy(), ro)
    if columns:
        cof, _ = oracle.gradient_permutation(oracle.nnz_histogram(A.rows, A.cols, rp, co, 1), 77, 1)
        np.testing.assert_array_equal(cperm.cpu().numpy(), cof)
    h = maxe.from_csr(Ad, rperm, cperm)
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    got = h.csr()
    np.testing.assert_array_equal(got[0].cpu().numpy(), nrp)
    np.testing.assert_array_equal(got[1].cpu().numpy(), nco)
    x = W.vector(2, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
    yo = oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())
    assert rel_l2(maxe.maxe_spmv(h, x).cpu().numpy(), yo) <= TOL[dtype]
    H, cnt = maxe.maxe_nnz_entropy(h, 64, 64)
    Ho, cnto = oracle.nnz_entropy(A.rows, A.cols, nrp, nco, 64, 64)
    np.testing.assert_array_equal(cnt.cpu().numpy(), cnto)
    assert H == pytest.approx(Ho, rel=1e-12)


def test_gradient_shuffle_spreads_clustered_heavy_rows():
    """Section 5: heavy rows clustered at the top leave most row bins light; the
    gradient cut plus riffle spreads them over the first half, and the row-bin
    entropy rises towards log2(bins)."""
    A = W.clustered_heavy(11, n=1 << 16, heavy_frac=0.05, heavy_len=400, dtype="f32").to("cuda")
    H0, _ = maxe.maxe_nnz_entropy(maxe.from_csr(A), 64, 1)
    rperm, _ = maxe.gradient_perms(A, 1)
    H1, _ = maxe.maxe_nnz_entropy(maxe.from_csr(A, rperm, None), 64, 1)
    assert H1 > H0 + 0.5
    assert H1 <= 6.0 + 1e-12


def test_gradient_invalid_arguments():
    h = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        maxe.maxe_gradient_permutation(h, 0, 2)
    with pytest.raises(RuntimeError):
        maxe.maxe_nnz_histogram(W.laplacian5(4, "f32").to("cuda"), 2)
