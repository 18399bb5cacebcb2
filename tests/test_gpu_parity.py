"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Permutations, permuted CSR arrays and histogram counts must be bit-exact.
Products must be within the relative-L2 tolerances of the FP64 oracle:
1e-12 (FP64 values), 1e-5 (FP32), 2e-3 (BF16 values, FP32 accumulation).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import EDGE_KINDS, TOL, code, edge_matrix, handle_arrays, oracle_permuted, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)
    yield
    torch.cuda.synchronize()
    assert maxe.maxe_device_status() == maxe.MAXE_OK


# ------------------------------------------------------------- permutation

@pytest.mark.parametrize("n", [1, 2, 3, 31, 1000, 4095, 4096, 4097, 100003, 1 << 20])
@pytest.mark.parametrize("tag", [0, 1])
def test_build_permutation_bit_exact(n, tag):
    seed = 2308 + n
    got = maxe.maxe_build_permutation(seed, n, tag).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.build_permutation(seed, n, tag))


def test_build_permutation_large_seed_and_zero():
    got = maxe.maxe_build_permutation(2**64 - 1, 5000, 1).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.build_permutation(2**64 - 1, 5000, 1))
    assert maxe.maxe_build_permutation(1, 0, 0).numel() == 0


def test_invert_gather_scatter_bit_exact():
    p = maxe.maxe_build_permutation(9, 77777, 0)
    pn = p.cpu().numpy()
    np.testing.assert_array_equal(maxe.maxe_invert_permutation(p).cpu().numpy(), oracle.invert_permutation(pn))
    for dt in (torch.float64, torch.float32, torch.bfloat16):
        x = torch.randn(77777, device="cuda").to(dt)
        g = maxe.maxe_permute_gather(p, x)
        s = maxe.maxe_permute_scatter(p, x)
        assert torch.equal(g, x[p.long()])
        ref = torch.empty_like(x)
        ref[p.long()] = x
        assert torch.equal(s, ref)
    x = W.vector(3, 77777, "f64", "cuda")
    np.testing.assert_array_equal(maxe.maxe_permute_gather(p, x).cpu().numpy(), oracle.gather(pn, x.cpu().numpy()))
    np.testing.assert_array_equal(maxe.maxe_permute_scatter(p, x).cpu().numpy(), oracle.scatter(pn, x.cpu().numpy()))


# ------------------------------------------------------------- permute_csr

def _perms(A, seed, mode):
    if mode == "plain":
        return None, None
    r = maxe.maxe_build_permutation(seed, A.rows, 0)
    c = maxe.maxe_build_permutation(seed, A.cols, 1) if mode == "rc" else None
    return r, c


@pytest.mark.parametrize("kind", EDGE_KINDS)
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("mode", ["plain", "r", "rc"])
def test_permute_csr_bit_exact_edges(kind, dtype, mode):
    A = edge_matrix(kind, dtype, seed=len(kind))
    rperm, cperm = _perms(A, 77, mode)
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, validate=True)
    got = handle_arrays(h)
    ref = oracle_permuted(A, rperm, cperm)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_permute_csr_bit_exact_blockdiag_and_laplacian(dtype):
    for A in (W.blockdiag(2308, dtype=dtype), W.laplacian5(300, dtype)):
        rperm, cperm = _perms(A, 5, "rc")
        h = maxe.from_csr(A.to("cuda"), rperm, cperm)
        for g, r in zip(handle_arrays(h), oracle_permuted(A, rperm, cperm)):
            np.testing.assert_array_equal(g, r)


def test_permute_csr_bit_exact_powerlaw_full_size():
    """1M-row power-law matrix (Zipf(1.5) rows capped at 1000, Gaussian columns)."""
    A = W.powerlaw(2308, device="cuda")
    rperm, cperm = _perms(A, 2308, "rc")
    h = maxe.from_csr(A, rperm, cperm)
    for g, r in zip(handle_arrays(h), oracle_permuted(A.to("cpu"), rperm, cperm)):
        np.testing.assert_array_equal(g, r)


def test_permute_csr_validate_rejects_bad_perm():
    A = edge_matrix("ragged", "f32").to("cuda")
    bad = torch.zeros(A.rows, dtype=torch.int32, device="cuda")
    with pytest.raises(maxe.MaxeError) as e:
        maxe.from_csr(A, bad, None, validate=True)
    assert e.value.status == maxe.MAXE_ERR_INVALID


# ---------------------------------------------------------------- products

@pytest.mark.parametrize("kind", EDGE_KINDS)
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("items16", [False, True])
def test_spmv_edges_original_and_permuted_space(kind, dtype, items16):
    A = edge_matrix(kind, dtype, seed=3)
    rperm, cperm = _perms(A, 11, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, items16=items16)
    assert h.items_per_lane() == (16 if items16 else 8)
    x = W.vector(5, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
    rp, co, va = A.numpy()
    y = maxe.maxe_spmv(h, x)  # y = A x through Eq. 1
    yo = oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())
    assert rel_l2(y.cpu().numpy(), yo) <= TOL[dtype]
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    xp = x[cperm.long()]
    yp = maxe.maxe_spmv(h, xp, permuted=True)  # y' = A' x'
    ypo = oracle.spmv(A.rows, nrp, nco, nva, code(dtype), xp.cpu().numpy())
    assert rel_l2(yp.cpu().numpy(), ypo) <= TOL[dtype]
    if A.rows:
        np.testing.assert_array_equal(yp.cpu().numpy()[torch.argsort(rperm).cpu().numpy()], y.cpu().numpy())


@pytest.mark.parametrize("case", ["ragged", "empty_nnz", "rect_wide", "rect_tall", "laplacian_xslice"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("pinned", [True, False])
def test_spmv_host_buffers_equal_the_device_call(case, dtype, pinned):
    """maxe_spmv_host (copy in, product, copy out, one stream) gives the bits of
    maxe_spmv on device vectors in both spaces, and the oracle's product."""
    A = W.laplacian5(300, dtype) if case == "laplacian_xslice" else edge_matrix(case, dtype, seed=7)
    rperm, cperm = _perms(A, 5, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, xslice=case == "laplacian_xslice")
    vt = torch.float64 if dtype == "f64" else torch.float32
    x = W.vector(9, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    got = {}
    for permuted in (False, True):
        xh = x.cpu()
        yh = torch.full((A.rows,), float("nan"), dtype=vt)
        if pinned:
            xh, yh = xh.pin_memory(), yh.pin_memory()
        xd = torch.full_like(x, float("nan"))
        yd = torch.empty(A.rows, dtype=vt, device="cuda")
        assert maxe.maxe_spmv_host(h, xh, yh, xd, yd, permuted=permuted, stream=st) is yh
        st.synchronize()
        ref = maxe.maxe_spmv(h, x, permuted=permuted)
        np.testing.assert_array_equal(yh.numpy(), ref.cpu().numpy())
        got[permuted] = yh.numpy().copy()
    rp, co, va = A.numpy()
    assert rel_l2(got[False], oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())) <= TOL[dtype]
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    assert rel_l2(got[True], oracle.spmv(A.rows, nrp, nco, nva, code(dtype), x.cpu().numpy())) <= TOL[dtype]


@pytest.mark.parametrize("shape", [(0, 5), (5, 0), (0, 0)])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_zero_row_and_zero_column_matrices(shape, dtype):
    """Degenerate shapes (no rows or no columns, so no nonzeros): every product
    is an empty or an all-zero vector, in both spaces and through every entry
    point; x holds no element when there are no columns and is never read."""
    M, N = shape
    A = W.from_lengths(1, [0] * M, N, dtype)
    rperm, cperm = _perms(A, 3, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, coo=True)
    vt = torch.float64 if dtype == "f64" else torch.float32
    x = torch.zeros(N, dtype=vt, device="cuda")
    for permuted in (False, True):
        y = torch.full((M,), float("nan"), dtype=vt, device="cuda")
        maxe.maxe_spmv(h, x, y, permuted=permuted)
        assert torch.equal(y, torch.zeros_like(y))
        y = torch.full((M,), float("nan"), dtype=vt, device="cuda")
        maxe.maxe_coo_spmv(h, x, y, permuted=permuted)
        assert torch.equal(y, torch.zeros_like(y))
        for k in (3, 16):
            Y = torch.full((M, k), float("nan"), dtype=vt, device="cuda")
            maxe.maxe_spmm(h, torch.zeros(N, k, dtype=vt, device="cuda"), Y, permuted=permuted)
            assert torch.equal(Y, torch.zeros_like(Y))
        yh = torch.full((M,), float("nan"), dtype=vt)
        maxe.maxe_spmv_host(h, x.cpu(), yh, torch.empty(N, dtype=vt, device="cuda"),
                            torch.empty(M, dtype=vt, device="cuda"), permuted=permuted)
        torch.cuda.synchronize()
        assert torch.equal(yh, torch.zeros_like(yh))


def test_spmv_host_rejects_device_tensors_and_wrong_lengths():
    A = edge_matrix("ragged", "f32", seed=7)
    h = maxe.from_csr(A.to("cuda"))
    xd = torch.zeros(A.cols, device="cuda")
    yd = torch.zeros(A.rows, device="cuda")
    with pytest.raises(ValueError):
        maxe.maxe_spmv_host(h, xd, yd.cpu(), xd, yd)
    with pytest.raises(ValueError):
        maxe.maxe_spmv_host(h, xd.cpu()[:-1], yd.cpu(), xd, yd)
    with pytest.raises(TypeError):
        maxe.maxe_spmv_host(h, xd.cpu().double(), yd.cpu(), xd, yd)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("mode", ["plain", "rc"])
def test_spmv_laplacian_and_blockdiag(dtype, mode):
    for A in (W.laplacian5(700, dtype), W.blockdiag(2308, dtype=dtype)):
        rperm, cperm = _perms(A, 1, mode)
        h = maxe.from_csr(A.to("cuda"), rperm, cperm)
        x = W.vector(8, A.cols, "f64" if dtype == "f64" else "f32", "cuda")
        rp, co, va = A.numpy()
        yo = oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())
        assert rel_l2(maxe.maxe_spmv(h, x).cpu().numpy(), yo) <= TOL[dtype]


def test_spmv_laplacian_closed_form_ones():
    n = 257
    A = W.laplacian5(n, "f32").to("cuda")
    rperm, cperm = _perms(A, 4, "rc")
    h = maxe.from_csr(A, rperm, cperm)
    y = maxe.maxe_spmv(h, torch.ones(n * n, device="cuda")).cpu().numpy().reshape(n, n)
    ref = np.zeros((n, n))
    ref[0, :] += 1
    ref[-1, :] += 1
    ref[:, 0] += 1
    ref[:, -1] += 1
    np.testing.assert_array_equal(y, ref)  # small integers: exact in FP32 whatever the order


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 16, 33, 64])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("lanes", ["passes", "lanes", "rows", "rows_pf"])
def test_spmm_against_oracle(k, dtype, lanes):
    A = edge_matrix("ragged", dtype, seed=k)
    rperm, cperm = _perms(A, k, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, spmm_lanes=lanes == "lanes", spmm_rows=lanes.startswith("rows"),
                      spmm_rows_pf=lanes == "rows_pf")
    assert h.spmm_lanes() == (lanes == "lanes") and h.spmm_rows() == lanes.startswith("rows")
    assert h.spmm_rows_prefetch() == (lanes == "rows_pf")
    X = W.matrix_rhs(k, A.cols, k, "f64" if dtype == "f64" else "f32", "cuda")
    rp, co, va = A.numpy()
    Yo = oracle.spmm(A.rows, rp, co, va, code(dtype), X.cpu().numpy())
    assert rel_l2(maxe.maxe_spmm(h, X).cpu().numpy(), Yo) <= TOL[dtype]
    # permuted space, and leading dimensions larger than k
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    Xp = X[cperm.long()]
    Xbig = torch.zeros(A.cols, k + 3, dtype=X.dtype, device="cuda")
    Xbig[:, :k] = Xp
    Ybig = torch.full((A.rows, k + 5), 7.0, dtype=X.dtype, device="cuda")
    maxe.maxe_spmm(h, Xbig[:, :k], Ybig[:, :k], permuted=True)
    Ypo = oracle.spmm(A.rows, nrp, nco, nva, code(dtype), Xp.cpu().numpy())
    assert rel_l2(Ybig[:, :k].cpu().numpy(), Ypo) <= TOL[dtype]
    assert torch.all(Ybig[:, k:] == 7.0)
    # leading dimensions padded to whole vectors: the tail column group is read
    # as a full vector (padding ignored) and written column by column
    kp = (k + 3) // 4 * 4
    Xpad = torch.full((A.cols, kp), float("nan"), dtype=X.dtype, device="cuda")
    Xpad[:, :k] = Xp
    Ypad = torch.full((A.rows, kp), 5.0, dtype=X.dtype, device="cuda")
    maxe.maxe_spmm(h, Xpad[:, :k], Ypad[:, :k], permuted=True)
    assert rel_l2(Ypad[:, :k].cpu().numpy(), Ypo) <= TOL[dtype]
    assert torch.all(Ypad[:, k:] == 5.0)


@pytest.mark.parametrize("kind", ["long_rows", "empty_runs", "unit_rows"])
@pytest.mark.parametrize("lanes", ["passes", "lanes", "rows", "rows_pf"])
def test_spmm_columns_match_spmv(kind, lanes):
    """Every column of an SpMM, and the SpMV of that column, are each within the
    FP32 bound of the FP64 oracle (the two kernels sum in different orders;
    rows here reach 70,000 entries)."""
    A = edge_matrix(kind, "f32", seed=2)
    rperm, cperm = _perms(A, 3, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, spmm_lanes=lanes == "lanes", spmm_rows=lanes.startswith("rows"),
                      spmm_rows_pf=lanes == "rows_pf")
    X = W.matrix_rhs(4, A.cols, 12, "f32", "cuda")
    Y = maxe.maxe_spmm(h, X)
    rp, co, va = A.numpy()
    for c in range(12):
        y = maxe.maxe_spmv(h, X[:, c].contiguous())
        ref = oracle.spmv(A.rows, rp, co, va, code("f32"), X[:, c].cpu().numpy())
        assert rel_l2(Y[:, c].cpu().numpy(), ref) <= TOL["f32"]
        assert rel_l2(y.cpu().numpy(), ref) <= TOL["f32"]


def test_products_are_deterministic():
    A = W.powerlaw(7, n=200000, device="cuda")
    h = maxe.from_csr(A, *_perms(A, 7, "rc"))
    x = W.vector(1, A.cols, "f32", "cuda")
    y1 = maxe.maxe_spmv(h, x)
    y2 = maxe.maxe_spmv(h, x)
    assert torch.equal(y1, y2)
    h2 = maxe.from_csr(A, *_perms(A, 7, "rc"))
    assert torch.equal(maxe.maxe_spmv(h2, x), y1)
    # the autotuned handle gives the oracle's result whichever variant it picks
    h3 = maxe.from_csr(A, *_perms(A, 7, "rc"), autotune=True)
    assert h3.items_per_lane() in (8, 16)
    assert rel_l2(maxe.maxe_spmv(h3, x).cpu().numpy(), y1.cpu().numpy()) <= 1e-6


# ----------------------------------------------------------------- entropy

@pytest.mark.parametrize("kind", ["ragged", "empty_runs", "long_rows", "rect_wide", "rect_tall", "unit_rows"])
@pytest.mark.parametrize("grid", [(1, 1), (2, 2), (8, 8), (3, 7), (64, 64)])
def test_entropy_counts_bit_exact(kind, grid):
    A = edge_matrix(kind, "f32", seed=1)
    gr, gc = min(grid[0], A.rows), min(grid[1], A.cols)
    for mode in ("plain", "rc"):
        rperm, cperm = _perms(A, 2, mode)
        h = maxe.from_csr(A.to("cuda"), rperm, cperm)
        nrp, nco, _ = oracle_permuted(A, rperm, cperm)
        H, cnt = maxe.maxe_nnz_entropy(h, gr, gc)
        Ho, co = oracle.nnz_entropy(A.rows, A.cols, nrp, nco, gr, gc)
        np.testing.assert_array_equal(cnt.cpu().numpy(), co)
        assert H == pytest.approx(Ho, rel=1e-12, abs=1e-15)


def test_entropy_wide_grids_and_bases():
    A = edge_matrix("ragged", "f64", seed=4)
    h = maxe.from_csr(A.to("cuda"), *_perms(A, 9, "rc"))
    nrp, nco, _ = oracle_permuted(A, *(_perms(A, 9, "rc")))
    for gr, gc, base in [(A.rows, 1, 2.0), (1, A.cols, 2.0), (A.rows, 7, math.e), (500, 500, 10.0), (1, 1, 2.0)]:
        H, cnt = maxe.maxe_nnz_entropy(h, gr, gc, base)
        Ho, co = oracle.nnz_entropy(A.rows, A.cols, nrp, nco, gr, gc, base)
        np.testing.assert_array_equal(cnt.cpu().numpy(), co)
        assert H == pytest.approx(Ho, rel=1e-12, abs=1e-15)


def test_entropy_rises_under_permutation_on_blockdiag():
    """Section 5: after a row+column permutation the 2-D histogram of a
    block-diagonal matrix is close to uniform, so H approaches log2(bins)."""
    A = W.blockdiag(2308, dtype="f64").to("cuda")
    H0, _ = maxe.maxe_nnz_entropy(maxe.from_csr(A), 16, 16)
    H1, _ = maxe.maxe_nnz_entropy(maxe.from_csr(A, *_perms(A, 1, "rc")), 16, 16)
    assert H0 < 5.0 and 7.9 < H1 <= 8.0  # measured by the oracle: 4.75 and 7.99


def test_entropy_rejects_bad_grid():
    A = edge_matrix("ragged", "f32").to("cuda")
    h = maxe.from_csr(A)
    for gr, gc, b in [(0, 1, 2.0), (A.rows + 1, 1, 2.0), (1, A.cols + 1, 2.0), (1, 1, 1.0)]:
        with pytest.raises(maxe.MaxeError) as e:
            maxe.maxe_nnz_entropy(h, gr, gc, b)
        assert e.value.status == maxe.MAXE_ERR_INVALID


# --------------------------------------------------------- power iteration

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_power_iteration_matches_oracle(dtype):
    n = 64
    A = W.laplacian5(n, dtype)
    rperm, cperm = _perms(A, 3, "rc")
    h = maxe.from_csr(A.to("cuda"), rperm, cperm)
    v0 = W.vector(4, n * n, dtype, "cuda")
    lam, v = maxe.maxe_power_iteration(h, v0, 20)
    rp, co, va = A.numpy()
    lo, vo = oracle.power_iteration(n * n, rp, co, va, code(dtype), v0.cpu().numpy(), 20)
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert lam == pytest.approx(lo, rel=tol)
    assert rel_l2(v.cpu().numpy(), vo) <= (1e-11 if dtype == "f64" else 1e-4)
    assert lam < 4 + 4 * math.cos(math.pi / (n + 1))


@pytest.mark.parametrize("xslice", [False, True])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_power_iteration_matches_oracle_step_by_step(dtype, xslice):
    """The Rayleigh quotient of every iterate equals the oracle's, step by step
    (FP64 within 1e-12, FP32 within 1e-5), on a permuted Laplacian and on a
    permuted power-law matrix; on the Laplacian it also rises monotonically and
    stays below its largest eigenvalue 4 + 4 cos(pi / (n + 1))."""
    n = 64
    for A in (W.laplacian5(n, dtype), W.powerlaw(11, n=20000, dtype=dtype)):
        M = A.rows
        rperm, cperm = _perms(A, 5, "rc")
        h = maxe.from_csr(A.to("cuda"), rperm, cperm, xslice=xslice)
        v0 = W.vector(6, M, dtype, "cuda")
        steps = 25
        lam, v, hist = maxe.maxe_power_iteration(h, v0, steps, history=True)
        rp, co, va = A.numpy()
        lo, vo, ho = oracle.power_iteration(M, rp, co, va, code(dtype), v0.cpu().numpy(), steps, history=True)
        tol = 1e-12 if dtype == "f64" else 1e-5
        assert hist.shape == (steps,) and hist[-1] == lam
        np.testing.assert_allclose(hist, ho, rtol=tol, atol=tol * np.abs(ho).max())
        if M == n * n:
            assert (np.diff(ho) >= -1e-12).all() and ho[-1] < 4 + 4 * math.cos(math.pi / (n + 1))
        h.close()


# ------------------------------------------------------------- host checks

def test_invalid_arguments_are_rejected():
    A = edge_matrix("ragged", "f32").to("cuda")
    h = maxe.from_csr(A)
    lib = maxe.load()
    import ctypes
    assert lib.maxe_spmm(ctypes.c_void_p(h.ptr), 0, None, 1, None, 1, 0, None) == maxe.MAXE_ERR_INVALID
    assert lib.maxe_spmm(ctypes.c_void_p(h.ptr), 65, None, 65, None, 65, 0, None) == maxe.MAXE_ERR_INVALID
    assert lib.maxe_spmv(ctypes.c_void_p(h.ptr), None, None, 0, None) == maxe.MAXE_ERR_INVALID
    assert lib.maxe_build_permutation(1, -1, 0, None, None, None) == maxe.MAXE_ERR_INVALID
    assert lib.maxe_build_permutation(1, 5, 2, None, None, None) == maxe.MAXE_ERR_INVALID
    assert lib.maxe_handle_destroy(None) == maxe.MAXE_OK


# ------------------------------------------- equal-rows partition (Section 5)

@pytest.mark.parametrize("kind", EDGE_KINDS + ["clustered"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_equal_rows_partition_products(kind, dtype):
    """The fixed equal-rows split gives the oracle's products (SpMV, both SpMM
    paths) in the original and the permuted space."""
    A = (W.clustered_heavy(5, n=20000, heavy_len=900, dtype=dtype) if kind == "clustered"
         else edge_matrix(kind, dtype, seed=8))
    rperm, cperm = _perms(A, 13, "rc")
    rp, co, va = A.numpy()
    vd = "f64" if dtype == "f64" else "f32"
    x = W.vector(3, A.cols, vd, "cuda")
    X = W.matrix_rhs(3, A.cols, 6, vd, "cuda")
    yo = oracle.spmv(A.rows, rp, co, va, code(dtype), x.cpu().numpy())
    Yo = oracle.spmm(A.rows, rp, co, va, code(dtype), X.cpu().numpy())
    for items16 in (False, True):
        for lanes in (False, True):
            h = maxe.from_csr(A.to("cuda"), rperm, cperm, equal_rows=True, items16=items16, spmm_lanes=lanes)
            assert rel_l2(maxe.maxe_spmv(h, x).cpu().numpy(), yo) <= TOL[dtype]
            assert rel_l2(maxe.maxe_spmm(h, X).cpu().numpy(), Yo) <= TOL[dtype]
    nrp, nco, nva = oracle_permuted(A, rperm, cperm)
    h = maxe.from_csr(A.to("cuda"), rperm, cperm, equal_rows=True)
    xp = x[cperm.long()]
    ypo = oracle.spmv(A.rows, nrp, nco, nva, code(dtype), xp.cpu().numpy())
    assert rel_l2(maxe.maxe_spmv(h, xp, permuted=True).cpu().numpy(), ypo) <= TOL[dtype]


def test_equal_rows_partition_unpermuted_and_deterministic():
    A = W.clustered_heavy(9, n=50000, heavy_len=2000, dtype="f32").to("cuda")
    x = W.vector(4, A.cols, "f32", "cuda")
    h = maxe.from_csr(A, equal_rows=True)
    rp, co, va = A.numpy()
    yo = oracle.spmv(A.rows, rp, co, va, code("f32"), x.cpu().numpy())
    y1 = maxe.maxe_spmv(h, x)
    assert rel_l2(y1.cpu().numpy(), yo) <= TOL["f32"]
    assert torch.equal(maxe.maxe_spmv(h, x), y1)


# ------------------------------------- hierarchical 2-D entropy (Section 5)

@pytest.mark.parametrize("grid,L", [((64, 64), 1), ((64, 64), 2), ((64, 64), 4), ((64, 64), 8), ((37, 53), 5),
                                    ((512, 512), 64), ((3000, 7), 7), ((1, 1), 1)])
def test_entropy_levels_against_oracle(grid, L):
    A = edge_matrix("ragged", "f32", seed=6)
    gr, gc = min(grid[0], A.rows), min(grid[1], A.cols)
    for mode in ("plain", "rc"):
        h = maxe.from_csr(A.to("cuda"), *_perms(A, 5, mode))
        H, cnt = maxe.maxe_nnz_entropy(h, gr, gc)
        for base in (2.0, math.e):
            lv = maxe.maxe_entropy_levels(cnt, L, base).cpu().numpy()
            ref = oracle.entropy_levels(cnt.cpu().numpy(), L, base)
            np.testing.assert_allclose(lv, ref, rtol=1e-12, atol=1e-15)
        if L == 1:
            assert lv[0, 0] == pytest.approx(math.log(2) * H, rel=1e-12, abs=1e-15)


def test_entropy_levels_permutation_flattens_the_map():
    """Section 5: on a block-diagonal matrix the per-block entropies are uneven
    (diagonal blocks far below log2 of their cell count); after row+column
    permutation every block is within sampling noise of it (about 1,450 entries
    over 256 cells here: an expected deficit near 0.13 bit)."""
    A = W.blockdiag(2308, dtype="f64").to("cuda")
    L, g = 4, 64
    _, c0 = maxe.maxe_nnz_entropy(maxe.from_csr(A), g, g)
    _, c1 = maxe.maxe_nnz_entropy(maxe.from_csr(A, *_perms(A, 3, "rc")), g, g)
    m0 = maxe.maxe_entropy_levels(c0, L).cpu().numpy()
    m1 = maxe.maxe_entropy_levels(c1, L).cpu().numpy()
    full = math.log2((g // L) ** 2)
    assert m1.min() > full - 0.25 and m1.max() <= full + 1e-12
    assert m1.max() - m1.min() < 0.15 and m0.max() - m0.min() > 0.3
    assert m0.min() < m1.min() - 1.0


def test_entropy_levels_rejects_bad_split():
    cnt = torch.ones(4, 4, dtype=torch.int64, device="cuda")
    for L in (0, 5):
        with pytest.raises(RuntimeError):
            maxe.maxe_entropy_levels(cnt, L)
