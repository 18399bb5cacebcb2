"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published test vector, a
library routine the paper names or an independent library routine, a closed
form, brute force on a tiny dense matrix, or an invariant the paper states.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats
import torch

import oracle
from paper_2308_00106_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_of(M, N, rowptr, col, val_f64):
    A = np.zeros((M, N), dtype=np.float64)
    for i in range(M):
        for t in range(rowptr[i], rowptr[i + 1]):
            A[i, col[t]] += val_f64[t]
    return A


def decode(val, dtype):
    """Stored values as float64, decoded with numpy casts (independent of oracle.c)."""
    if dtype == oracle.BF16:
        return (val.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return val.astype(np.float64)


def small_csr(seed, M, N, dtype="f64", density=0.3, empty_rows=True):
    g = np.random.default_rng(seed)
    lengths = g.binomial(N, density, M)
    if empty_rows and M > 2:
        lengths[g.integers(0, M, max(1, M // 5))] = 0
    A = W.from_lengths(seed, lengths, N, dtype)
    return A


# --------------------------------------------------------------- permutation

def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for _, tag, i, hexv in rows:
        assert oracle.key(0, int(tag), int(i)) == int(hexv, 16)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 4097])
def test_permutation_sorts_keys_like_numpy(n):
    seed = 12345 + n
    perm = oracle.build_permutation(seed, n, 0)
    keys = np.array([oracle.key(seed, 0, i) for i in range(n)], dtype=np.uint64)
    # independent library sort: stable argsort on the keys, ties by index
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable").astype(np.int32))
    assert sorted(perm.tolist()) == list(range(n))


def test_permutation_rows_and_cols_streams_differ():
    a = oracle.build_permutation(7, 512, 0)
    b = oracle.build_permutation(7, 512, 1)
    c = oracle.build_permutation(8, 512, 0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_permutation_uniform_positions():
    """Section 3 asks for a uniformly random permutation: over many seeds, every
    element lands in every position equally often (chi-square)."""
    n, seeds = 8, 4000
    hits = np.zeros((n, n), dtype=np.int64)
    for s in range(seeds):
        p = oracle.build_permutation(s, n, s & 1)
        hits[p, np.arange(n)] += 1
    chi = scipy.stats.chisquare(hits.ravel(), np.full(n * n, seeds / n))
    assert chi.pvalue > 1e-4, chi


def test_invert_permutation_and_rejects_non_bijection():
    p = oracle.build_permutation(3, 100, 1)
    inv = oracle.invert_permutation(p)
    np.testing.assert_array_equal(inv[p], np.arange(100))
    with pytest.raises(ValueError):
        oracle.invert_permutation(np.array([0, 0, 1], dtype=np.int32))


def test_gather_scatter_are_inverse():
    p = oracle.build_permutation(5, 50, 0)
    x = np.random.default_rng(0).standard_normal(50)
    np.testing.assert_array_equal(oracle.gather(p, x), x[p])
    np.testing.assert_array_equal(oracle.scatter(p, oracle.gather(p, x)), x)


# --------------------------------------------------------------- permute_csr

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", [(1, 1), (17, 23), (64, 64), (40, 9)])
def test_permute_csr_matches_dense_fancy_indexing(dtype, shape):
    M, N = shape
    A = small_csr(M * 31 + N, M, N, dtype)
    code = W.DTYPE_CODE[dtype]
    rp, co, va = A.numpy()
    rperm = oracle.build_permutation(11, M, 0)
    cperm = oracle.build_permutation(11, N, 1)
    ro, cn, vn = oracle.permute_csr(M, N, rp, co, va, code, rperm, cperm)
    D = dense_of(M, N, rp, co, decode(va, code))
    Dp = dense_of(M, N, ro, cn, decode(vn, code))
    # Eq. 1: A' = P_r A P_c with perm[new] = old  <=>  A'[i', j'] = A[rperm[i'], cperm[j']]
    np.testing.assert_array_equal(Dp, D[np.ix_(rperm, cperm)])
    assert ro[-1] == rp[-1]  # nnz preserved
    for i in range(M):  # ascending columns, row lengths carried with the row
        seg = cn[ro[i]:ro[i + 1]]
        assert np.all(np.diff(seg) > 0)
        assert ro[i + 1] - ro[i] == rp[rperm[i] + 1] - rp[rperm[i]]


def test_permute_csr_inverse_restores_bit_exactly():
    A = small_csr(99, 50, 60, "bf16")
    rp, co, va = A.numpy()
    rperm = oracle.build_permutation(1, 50, 0)
    cperm = oracle.build_permutation(1, 60, 1)
    r1, c1, v1 = oracle.permute_csr(50, 60, rp, co, va, 2, rperm, cperm)
    r2, c2, v2 = oracle.permute_csr(50, 60, r1, c1, v1, 2, oracle.invert_permutation(rperm),
                                    oracle.invert_permutation(cperm))
    np.testing.assert_array_equal(r2, rp)
    np.testing.assert_array_equal(c2, co)
    np.testing.assert_array_equal(v2.view(np.uint16), va.view(np.uint16))


def test_permute_csr_identity_sorts_unsorted_rows_stably():
    rowptr = np.array([0, 3, 3, 5], dtype=np.int32)
    col = np.array([4, 0, 2, 1, 0], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    r, c, v = oracle.permute_csr(3, 5, rowptr, col, val, 0)
    np.testing.assert_array_equal(r, rowptr)
    np.testing.assert_array_equal(c, [0, 2, 4, 0, 1])
    np.testing.assert_array_equal(v, [2.0, 3.0, 1.0, 5.0, 4.0])


# ---------------------------------------------------------------------- SpMV

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", [(1, 1), (5, 64), (64, 64), (33, 7)])
def test_spmv_matches_dense_brute_force(dtype, shape):
    M, N = shape
    A = small_csr(M + 7 * N, M, N, dtype, density=0.4)
    code = W.DTYPE_CODE[dtype]
    rp, co, va = A.numpy()
    x = np.random.default_rng(M).uniform(-1, 1, N)
    y = oracle.spmv(M, rp, co, va, code, x)
    D = dense_of(M, N, rp, co, decode(va, code))
    np.testing.assert_allclose(y, D @ x, rtol=1e-13, atol=1e-13)


def test_spmm_matches_dense_brute_force():
    A = small_csr(5, 40, 30, "f32", density=0.3)
    rp, co, va = A.numpy()
    X = np.random.default_rng(1).uniform(-1, 1, (30, 5))
    Y = oracle.spmm(40, rp, co, va, 1, X)
    D = dense_of(40, 30, rp, co, decode(va, 1))
    np.testing.assert_allclose(Y, D @ X, rtol=1e-13, atol=1e-13)
    rows = np.array([0, 39, 17])
    np.testing.assert_allclose(oracle.spmv_rows(rp, co, va, 1, X[:, 2], rows), (D @ X[:, 2])[rows], rtol=1e-13)


def test_spmv_empty_matrix_and_empty_rows():
    rowptr = np.zeros(4, dtype=np.int32)
    y = oracle.spmv(3, rowptr, np.zeros(0, np.int32), np.zeros(0), 0, np.ones(5))
    np.testing.assert_array_equal(y, np.zeros(3))


@pytest.mark.parametrize("n", [1, 2, 3, 16, 45])
def test_laplacian_closed_forms(n):
    L = W.laplacian5(n, "f64")
    rp, co, va = L.numpy()
    assert L.nnz == 5 * n * n - 4 * n
    # x = 1: interior rows sum to 0, edge rows to 1, corners to 2 (n > 1)
    y = oracle.spmv(n * n, rp, co, va, 0, np.ones(n * n)).reshape(n, n)
    missing = np.zeros((n, n))
    missing[0, :] += 1
    missing[-1, :] += 1
    missing[:, 0] += 1
    missing[:, -1] += 1
    np.testing.assert_array_equal(y, missing)
    # exact eigenvector sin(pi a/(n+1)) sin(pi b/(n+1)), lambda = 4 - 4 cos(pi/(n+1))
    a = np.arange(1, n + 1)
    v = np.outer(np.sin(np.pi * a / (n + 1)), np.sin(np.pi * a / (n + 1))).ravel()
    lam = 4 - 4 * math.cos(math.pi / (n + 1))
    np.testing.assert_allclose(oracle.spmv(n * n, rp, co, va, 0, v), lam * v, rtol=0, atol=1e-13)


def test_eq1_identity_unpermuted_product():
    A = small_csr(8, 70, 50, "f64")
    rp, co, va = A.numpy()
    rperm = oracle.build_permutation(21, 70, 0)
    cperm = oracle.build_permutation(21, 50, 1)
    ro, cn, vn = oracle.permute_csr(70, 50, rp, co, va, 0, rperm, cperm)
    x = np.random.default_rng(2).uniform(-1, 1, 50)
    yp = oracle.spmv(70, ro, cn, vn, 0, oracle.gather(cperm, x))
    np.testing.assert_allclose(oracle.scatter(rperm, yp), oracle.spmv(70, rp, co, va, 0, x), rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------------- entropy

def _hist_matrix(h):
    """CSR whose row lengths are the histogram h (one column)."""
    h = np.asarray(h, dtype=np.int64)
    N = max(int(h.max()), 1)
    rowptr = np.concatenate([[0], np.cumsum(h)]).astype(np.int32)
    col = np.concatenate([np.arange(k) for k in h]).astype(np.int32) if h.sum() else np.zeros(0, np.int32)
    return len(h), N, rowptr, col


def test_entropy_golden_closed_forms():
    for line in open(os.path.join(GOLDEN, "entropy_closed_forms.txt")):
        if line.startswith("#") or not line.strip():
            continue
        base, counts, H = [s.strip() for s in line.split(";")]
        h = [int(c) for c in counts.split(",")]
        M, N, rowptr, col = _hist_matrix(h)
        got, cnt = oracle.nnz_entropy(M, N, rowptr, col, M, 1, float(base))
        np.testing.assert_array_equal(cnt.ravel(), h)
        assert got == pytest.approx(float(H), abs=1e-15)


@pytest.mark.parametrize("g", [(1, 1), (2, 2), (4, 8), (16, 16)])
def test_entropy_uniform_grid_is_log2_bins(g):
    gr, gc = g
    n = 64
    # one entry in the top-left cell of every block: every bin has the same count
    rows, cols = [], []
    for i in range(n):
        for j in range(n):
            if i % (n // gr) == 0 and j % (n // gc) == 0:
                rows.append(i)
                cols.append(j)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    H, cnt = oracle.nnz_entropy(n, n, rowptr, np.array(cols, np.int32), gr, gc)
    assert np.all(cnt == 1)
    assert H == math.log2(gr * gc)  # exact for power-of-two bin counts


def test_entropy_special_cases_reduce_to_row_and_column_counts():
    A = small_csr(4, 30, 20, "f64")
    rp, co, va = A.numpy()
    _, cnt = oracle.nnz_entropy(30, 20, rp, co, 30, 1)
    np.testing.assert_array_equal(cnt.ravel(), np.diff(rp))  # per-row histogram = row lengths
    _, cnt = oracle.nnz_entropy(30, 20, rp, co, 1, 20)
    np.testing.assert_array_equal(cnt.ravel(), np.bincount(co, minlength=20))  # per-column = column counts
    H, cnt = oracle.nnz_entropy(30, 20, rp, co, 1, 1)
    assert H == 0.0 and cnt[0, 0] == A.nnz


@pytest.mark.parametrize("g", [(3, 5), (7, 7), (30, 20), (1, 13)])
def test_entropy_matches_scipy_and_dense_block_sums(g):
    gr, gc = g
    M, N = 30, 20
    A = small_csr(17, M, N, "f64", density=0.5)
    rp, co, va = A.numpy()
    H, cnt = oracle.nnz_entropy(M, N, rp, co, gr, gc)
    # block sums of the dense nonzero indicator, blocks cut at ceil(b*M/gr)
    D = dense_of(M, N, rp, co, np.ones(A.nnz)) != 0
    re = [-(-b * M // gr) for b in range(gr + 1)]
    ce = [-(-b * N // gc) for b in range(gc + 1)]
    blocks = np.array([[D[re[a]:re[a + 1], ce[b]:ce[b + 1]].sum() for b in range(gc)] for a in range(gr)])
    np.testing.assert_array_equal(cnt, blocks)
    # the paper computes H with scipy.stats.entropy (Section 4)
    assert H == pytest.approx(scipy.stats.entropy(cnt.ravel(), base=2), rel=1e-13, abs=1e-15)
    assert H <= math.log2(gr * gc) + 1e-12
    # natural-log reading of "scipy stats" default base
    He, _ = oracle.nnz_entropy(M, N, rp, co, gr, gc, math.e)
    assert He == pytest.approx(scipy.stats.entropy(cnt.ravel()), rel=1e-13, abs=1e-15)


def test_entropy_ignores_bin_order():
    """Section 5: entropy depends on the bin probabilities only, so permuting the
    rows with one bin per row leaves it unchanged."""
    A = small_csr(23, 40, 40, "f64")
    rp, co, va = A.numpy()
    H0, _ = oracle.nnz_entropy(40, 40, rp, co, 40, 1)
    ro, cn, _ = oracle.permute_csr(40, 40, rp, co, va, 0, oracle.build_permutation(2, 40, 0), None)
    H1, _ = oracle.nnz_entropy(40, 40, ro, cn, 40, 1)
    assert H1 == pytest.approx(H0, rel=1e-14)


def test_entropy_rejects_bad_grid():
    with pytest.raises(ValueError):
        oracle.nnz_entropy(4, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), 5, 1)


# ------------------------------------------------------------ power iteration

def test_power_iteration_diagonal_closed_form():
    d = np.array([1.0, -3.0, 10.0, 5.0, 2.0])
    rowptr = np.arange(6, dtype=np.int32)
    col = np.arange(5, dtype=np.int32)
    lam, v = oracle.power_iteration(5, rowptr, col, d, 0, np.ones(5), 60)
    assert lam == pytest.approx(10.0, rel=1e-12)
    assert abs(v[2]) == pytest.approx(1.0, rel=1e-12)


def test_power_iteration_laplacian_bounds_and_monotone():
    n = 12
    L = W.laplacian5(n, "f64")
    rp, co, va = L.numpy()
    v0 = np.random.default_rng(4).uniform(-1, 1, n * n)
    lam, v, hist = oracle.power_iteration(n * n, rp, co, va, 0, v0, 20, history=True)
    lam_max = 4 + 4 * math.cos(math.pi / (n + 1))
    assert lam < lam_max
    assert np.all(np.diff(hist) >= -1e-12)  # Rayleigh quotients of an SPD matrix never decrease
    assert hist[-1] == pytest.approx(lam, rel=1e-14)
