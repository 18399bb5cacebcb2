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


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_coo_spmv_matches_dense_and_any_triplet_order(dtype):
    A = small_csr(51, 45, 38, dtype, density=0.3)
    rp, co, va = A.numpy()
    row = oracle.csr_to_coo_rows(45, rp)
    np.testing.assert_array_equal(row, np.repeat(np.arange(45), np.diff(rp)))
    x = np.random.default_rng(3).uniform(-1, 1, 38)
    D = dense_of(45, 38, rp, co, decode(va, W.DTYPE_CODE[dtype]))
    y = oracle.coo_spmv(45, row, co, va, W.DTYPE_CODE[dtype], x)
    np.testing.assert_allclose(y, D @ x, rtol=1e-13, atol=1e-14)
    perm = np.random.default_rng(4).permutation(row.size)  # COO keeps no order
    y2 = oracle.coo_spmv(45, row[perm], co[perm], va[perm], W.DTYPE_CODE[dtype], x)
    np.testing.assert_allclose(y2, y, rtol=1e-13, atol=1e-14)
    # in CSR order the sums run in the same order as the CSR product: identical
    np.testing.assert_array_equal(y, oracle.spmv(45, rp, co, va, W.DTYPE_CODE[dtype], x))


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


# ------------------------------------------- hierarchical 2-D entropy (Section 5)

def test_entropy_levels_one_block_is_global_entropy():
    A = small_csr(31, 40, 36, "f64", density=0.4)
    rp, co, va = A.numpy()
    H, cnt = oracle.nnz_entropy(40, 36, rp, co, 8, 6)
    lv = oracle.entropy_levels(cnt, 1)
    assert lv.shape == (1, 1) and lv[0, 0] == pytest.approx(H, rel=1e-14)


@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_entropy_levels_uniform_counts_are_log2_cells(L):
    counts = np.full((16, 16), 3, dtype=np.int64)
    lv = oracle.entropy_levels(counts, L)
    assert np.all(lv == math.log2((16 // L) ** 2))  # exact: power-of-two cells per block


def test_entropy_levels_single_cell_and_empty_blocks_are_zero():
    counts = np.zeros((8, 8), dtype=np.int64)
    counts[0, 0] = 7  # block (0, 0) of a 2 x 2 split holds one nonzero cell
    counts[6, 1] = 2
    counts[7, 2] = 2  # block (1, 0): two equal cells -> 1 bit
    lv = oracle.entropy_levels(counts, 2)
    assert lv[0, 0] == 0.0 and lv[0, 1] == 0.0 and lv[1, 1] == 0.0
    assert lv[1, 0] == 1.0


@pytest.mark.parametrize("shape,L", [((13, 11), 3), ((32, 32), 4), ((9, 20), 9), ((64, 48), 8)])
def test_entropy_levels_match_scipy_on_numpy_blocks(shape, L):
    g = np.random.default_rng(shape[0] * 100 + L)
    counts = g.integers(0, 5, size=shape).astype(np.int64)
    counts[g.random(shape) < 0.3] = 0
    lv = oracle.entropy_levels(counts, L)
    gr, gc = shape
    re = [-(-a * gr // L) for a in range(L + 1)]
    ce = [-(-b * gc // L) for b in range(L + 1)]
    for a in range(L):
        for b in range(L):
            blk = counts[re[a]:re[a + 1], ce[b]:ce[b + 1]].ravel()
            want = scipy.stats.entropy(blk, base=2) if blk.sum() else 0.0
            assert lv[a, b] == pytest.approx(want, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("L", [2, 3, 5])
def test_entropy_levels_chain_rule(L):
    """H(cells) = H(blocks) + sum_b P(b) H(cells | b): the map and the block totals
    must recompose the global entropy, whatever the block edges."""
    g = np.random.default_rng(L)
    counts = g.integers(0, 9, size=(20, 15)).astype(np.int64)
    lv = oracle.entropy_levels(counts, L)
    Hg = oracle.entropy_levels(counts, 1)[0, 0]
    # block totals from the oracle's own edges, reconstructed as those of the L-split
    re = [-(-a * 20 // L) for a in range(L + 1)]
    ce = [-(-b * 15 // L) for b in range(L + 1)]
    tot = np.array([[counts[re[a]:re[a + 1], ce[b]:ce[b + 1]].sum() for b in range(L)] for a in range(L)], float)
    P = tot / tot.sum()
    Hb = scipy.stats.entropy(P.ravel(), base=2)
    assert Hg == pytest.approx(Hb + float((P * lv).sum()), rel=1e-13)


def test_entropy_levels_rejects_bad_split():
    with pytest.raises(ValueError):
        oracle.entropy_levels(np.ones((4, 4), np.int64), 5)
    with pytest.raises(ValueError):
        oracle.entropy_levels(np.ones((4, 4), np.int64), 0)


# ------------------------------- gradient-based permutations (Section 5, appendix)

def test_nnz_histogram_rows_and_columns():
    A = small_csr(41, 33, 27, "f64", density=0.35)
    rp, co, _ = A.numpy()
    np.testing.assert_array_equal(oracle.nnz_histogram(33, 27, rp, co, 0), np.diff(rp))
    np.testing.assert_array_equal(oracle.nnz_histogram(33, 27, rp, co, 1), np.bincount(co, minlength=27))


def _deck_from_perm(perm, seed, tag):
    """Undo the per-half random order with numpy's sort of the published
    SplitMix64 keys: deck[q] = perm[s + rank of q inside its half]."""
    n = perm.size
    half = (n + 1) // 2
    deck = np.empty(n, dtype=np.int64)
    for s, e in ((0, half), (half, n)):
        q = np.arange(s, e)
        keys = np.array([oracle.key(seed, tag, int(i)) for i in q], dtype=np.uint64)
        order = q[np.lexsort((q, keys))]  # positions sorted by (key, position)
        deck[order] = perm[s:e]
    return deck


@pytest.mark.parametrize("seed", [0, 5, 2**63 + 11])
def test_gradient_pivot_is_first_steepest_step(seed):
    g = np.random.default_rng(seed % 1000)
    for n in (2, 3, 17, 100, 501):
        h = g.integers(0, 4, n)  # small range: many tied gradients
        perm, pivot = oracle.gradient_permutation(h, seed, 0)
        assert pivot == int(np.argmax(np.abs(np.diff(h)))) + 1  # numpy argmax: first maximum
        assert np.array_equal(np.sort(perm), np.arange(n))


def test_gradient_riffle_at_middle_is_the_out_faro_shuffle():
    """A cut at n/2 makes the riffle a perfect out-shuffle (top card stays on
    top); eight out-shuffles restore a 52-card deck, a textbook fact."""
    h = np.array([7] * 26 + [2] * 26)
    for seed in (1, 2, 3):
        perm, pivot = oracle.gradient_permutation(h, seed, 1)
        assert pivot == 26
        deck = _deck_from_perm(perm, seed, 1)
        np.testing.assert_array_equal(deck[0::2], np.arange(26))
        np.testing.assert_array_equal(deck[1::2], np.arange(26, 52))
        p = np.arange(52)
        for r in range(1, 9):
            p = p[deck]
            assert np.array_equal(p, np.arange(52)) == (r == 8)  # order exactly 8


@pytest.mark.parametrize("n,cut", [(10, 3), (10, 7), (9, 1), (9, 8), (1000, 13), (1001, 990)])
def test_gradient_riffle_with_unequal_parts(n, cut):
    """Alternate cards while both parts last, then the longer part's remainder in order."""
    h = np.zeros(n, dtype=np.int64)
    h[:cut] = 50  # one step, at the cut
    perm, pivot = oracle.gradient_permutation(h, 77, 0)
    assert pivot == cut
    deck = _deck_from_perm(perm, 77, 0)
    m = min(cut, n - cut)
    np.testing.assert_array_equal(deck[0:2 * m:2], np.arange(m))
    np.testing.assert_array_equal(deck[1:2 * m:2], cut + np.arange(m))
    rest = np.arange(m, cut) if cut > n - cut else np.arange(cut + m, n)
    np.testing.assert_array_equal(deck[2 * m:], rest)


def test_gradient_degenerate_sizes_and_flat_histogram():
    assert oracle.gradient_permutation([], 3, 0)[0].size == 0
    perm, pivot = oracle.gradient_permutation([4], 3, 0)
    assert perm.tolist() == [0] and pivot == 1
    perm, pivot = oracle.gradient_permutation([2, 9], 3, 0)
    assert pivot == 1 and perm.tolist() == [0, 1]  # deck [0, 1], halves of one card each
    perm, pivot = oracle.gradient_permutation(np.full(40, 6), 3, 0)
    assert pivot == 1  # flat: every gradient ties at 0, the first wins


def test_gradient_halves_are_uniformly_permuted():
    """Each card of a half lands on each position of the half equally often over seeds."""
    n, trials = 8, 4000
    h = np.array([9, 9, 9, 9, 1, 1, 1, 1])
    pos = np.zeros((n, n))
    for seed in range(trials):
        perm, _ = oracle.gradient_permutation(h, seed, 0)
        pos[perm, np.arange(n)] += 1
    # cards of the first half of the deck [0, 4, 1, 5] stay in positions 0..3
    for card in (0, 4, 1, 5):
        assert pos[card, 4:].sum() == 0
        chi2 = ((pos[card, :4] - trials / 4) ** 2 / (trials / 4)).sum()
        assert chi2 < 16.3  # 3 d.o.f., p ~ 0.001


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
