"""GPU parity of the COO product (Section 2, triplets ROW, COL, VALUE): row
indices bit-exact, products within the FP tolerance of the FP64 oracle, in the
permuted and the original space, deterministic."""
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


def _perms(A, seed):
    return maxe.maxe_build_permutation(seed, A.rows, 0), maxe.maxe_build_permutation(seed, A.cols, 1)


def _chunk_edges(dtype, seed):
    """Row lengths around the 256-entry chunk and 8-entry lane sizes, runs of empty rows."""
    g = np.random.default_rng(seed)
    L = g.choice([0, 0, 1, 7, 8, 9, 255, 256, 257, 513, 2000], size=3000)
    return W.from_lengths(seed, L, 4000, dtype)


@pytest.mark.parametrize("kind", EDGE_KINDS + ["chunk_edges"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_coo_spmv_against_oracle(kind, dtype):
    A = _chunk_edges(dtype, 4) if kind == "chunk_edges" else edge_matrix(kind, dtype, seed=5)
    rperm, cperm = _perms(A, 21)
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, coo=True)
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    np.testing.assert_array_equal(h.coo_rows().cpu().numpy(), oracle.csr_to_coo_rows(A.rows, nrp))
    vd = "f64" if dtype == "f64" else "f32"
    x = W.vector(6, A.cols, vd, "cuda")
    xp = x[cperm.long()]
    yp = torch.full((A.rows,), float("nan"), dtype=x.dtype, device="cuda")  # every row must be written
    maxe.maxe_coo_spmv(h, xp, yp, permuted=True)
    ypo = oracle.coo_spmv(A.rows, oracle.csr_to_coo_rows(A.rows, nrp), nco, nva, code(dtype), xp.cpu().numpy())
    assert not torch.isnan(yp).any()
    assert rel_l2(yp.cpu().numpy(), ypo) <= TOL[dtype]
    rp, co, va = A.numpy()
    y = torch.full((A.rows,), float("nan"), dtype=x.dtype, device="cuda")
    maxe.maxe_coo_spmv(h, x, y)  # original space: gather x through cperm, scatter y through rperm
    assert not torch.isnan(y).any()
    assert rel_l2(y.cpu().numpy(), oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())) <= TOL[dtype]


def test_coo_matches_csr_and_is_deterministic():
    A = W.powerlaw(3, n=300000, device="cuda")
    h = maxe.from_csr(A, *_perms(A, 3), coo=True)
    x = W.vector(2, A.cols, "f32", "cuda")
    y1 = maxe.maxe_coo_spmv(h, x)
    assert torch.equal(maxe.maxe_coo_spmv(h, x), y1)
    assert rel_l2(y1.cpu().numpy(), maxe.maxe_spmv(h, x).cpu().numpy()) <= 1e-6
    rp, co, va = A.numpy()
    rows = np.random.default_rng(0).choice(A.rows, 3000, replace=False)
    ref = oracle.spmv_rows(rp, co, va, code("f32"), x.cpu().numpy(), rows)
    assert rel_l2(y1.cpu().numpy()[rows], ref) <= TOL["f32"]


def test_coo_single_long_row_spans_many_chunks():
    lengths = np.zeros(50, dtype=np.int64)
    lengths[[0, 20, 49]] = [3, 70000, 256]
    A = W.from_lengths(9, lengths, 80000, "f64")
    h = maxe.from_csr(A.to("cuda"), coo=True)
    x = W.vector(1, A.cols, "f64", "cuda")
    rp, co, va = A.numpy()
    y = maxe.maxe_coo_spmv(h, x)
    assert rel_l2(y.cpu().numpy(), oracle.spmv(A.rows, rp, co, va, code("f64"), x.cpu().numpy())) <= TOL["f64"]


def test_coo_long_runs_of_empty_rows():
    """Runs of empty rows longer than a warp (zeroed by the whole warp), at the
    start, in the middle and after the last entry."""
    lengths = np.zeros(300000, dtype=np.int64)
    lengths[[70000, 70001, 150000, 200000]] = [5, 300, 2, 40]
    A = W.from_lengths(4, lengths, 1000, "f32")
    rperm = maxe.maxe_build_permutation(3, A.rows, 0)
    h = maxe.from_csr(A.to("cuda"), rperm, None, coo=True)
    x = W.vector(2, A.cols, "f32", "cuda")
    for permuted in (False, True):
        y = torch.full((A.rows,), float("nan"), device="cuda")
        maxe.maxe_coo_spmv(h, x, y, permuted=permuted)
        assert not torch.isnan(y).any()
    rp, co, va = A.numpy()
    y = maxe.maxe_coo_spmv(h, x)
    assert rel_l2(y.cpu().numpy(), oracle.spmv(A.rows, rp, co, va, code("f32"), x.cpu().numpy())) <= TOL["f32"]


def test_coo_requires_the_flag():
    A = W.laplacian5(8, "f32").to("cuda")
    h = maxe.from_csr(A)
    with pytest.raises(RuntimeError):
        maxe.maxe_coo_spmv(h, torch.ones(A.cols, device="cuda"))
    with pytest.raises(RuntimeError):
        h.coo_rows()
