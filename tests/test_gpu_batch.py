"""Batched persistent launch (many matrices, uneven sizes, 1..k right-hand
sides) against the CPU oracle, and the determinism the serving loop relies on:
an item's result is bit-identical alone and in any mix."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_00106_gb300 import maxe
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import TOL, code, edge_matrix, oracle_permuted, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)
    yield
    torch.cuda.synchronize()
    assert maxe.maxe_device_status() == maxe.MAXE_OK


def _mats():
    """Uneven matrices of all three value types, with edge-case structure."""
    specs = [("ragged", "f32"), ("long_rows", "f32"), ("empty_runs", "bf16"), ("unit_rows", "f32"),
             ("rect_wide", "f64"), ("rect_tall", "bf16"), ("one", "f32"), ("empty_nnz", "f32")]
    out = [edge_matrix(kind, dt, seed=i + 1) for i, (kind, dt) in enumerate(specs)]
    out += [W.poisson_uniform(40 + i, 3000 * (i + 1), 8.0 + 7 * i, "f32") for i in range(4)]
    return out


KS = [1, 3, 16, 2, 5, 4, 1, 7, 1, 9, 2, 12]


def _setup(mats, ks, seed=1):
    items = []
    for i, (A, k) in enumerate(zip(mats, ks)):
        r = maxe.maxe_build_permutation(seed + i, A.rows, 0)
        c = maxe.maxe_build_permutation(seed + i, A.cols, 1)
        # SpMM kernels of one mix: items 0, 3, ... one row per lane group (the
        # default plan, X rows padded to 16 bytes); 1, 4, ... columns across
        # lanes; 2, 5, ... unpadded X rows, which the rows kernel cannot take,
        # so the default plan falls back to column passes
        h = maxe.from_csr(A.to("cuda"), r, c, spmm_lanes=(i % 3 == 1))
        kp = ((k + 3) // 4 * 4 if i % 3 != 2 else k) if k > 1 else 1
        Xb = torch.zeros(A.cols, kp, dtype=torch.float64 if A.dtype == "f64" else torch.float32, device="cuda")
        Xb[:, :k] = W.matrix_rhs(100 + i, A.cols, k, "f64" if A.dtype == "f64" else "f32", "cuda")
        items.append((A, h, r, c, Xb[:, :k]))
    return items


def _check_against_oracle(A, r, c, X, Y, scatter):
    """X is X' (permuted space).  Without scatter Y must be A' X'; with scatter
    Y = A X where X[cperm[j]] = X'[j] (Eq. 1)."""
    Xp = X.cpu().numpy()
    if scatter:
        rp, co, va = A.numpy()
        Xo = np.empty_like(Xp)
        Xo[c.cpu().numpy()] = Xp
        ref = oracle.spmm(A.rows, rp, co, va, code(A.dtype), Xo)
    else:
        nrp, nco, nva = oracle_permuted(A, r, c)
        ref = oracle.spmm(A.rows, nrp, nco, nva, code(A.dtype), Xp)
    assert rel_l2(Y.cpu().numpy(), ref) <= TOL[A.dtype]


@pytest.mark.parametrize("scatter", [False, True])
def test_batch_matches_oracle_per_item(scatter):
    mats = _mats()
    items = _setup(mats, KS)
    b = maxe.Batch(len(items))
    Ys = [torch.full((A.rows, X.stride(0)), float("nan"), dtype=X.dtype, device="cuda")[:, :X.shape[1]]
          for A, h, r, c, X in items]
    b.set([(h, X, Y, scatter) for (A, h, r, c, X), Y in zip(items, Ys)])
    b.run()
    torch.cuda.synchronize()
    for (A, h, r, c, X), Y in zip(items, Ys):
        _check_against_oracle(A, r, c, X, Y, scatter)


def test_batch_plans_pick_the_spmm_kernels():
    items = _setup(_mats(), KS)
    kinds = [h.batch_spmm_kernel() for A, h, r, c, X in items]
    assert kinds == ["rows" if i % 3 != 1 else "lanes" for i in range(len(items))]
    for A, h, r, c, X in items:
        h.close()


def test_batch_item_alone_equals_in_mix_bitwise():
    mats = _mats()
    items = _setup(mats, KS, seed=7)
    b = maxe.Batch(len(items))
    Ymix = [torch.empty((A.rows, X.stride(0)), dtype=X.dtype, device="cuda")[:, :X.shape[1]] for A, h, r, c, X in items]
    b.set([(h, X, Y, False) for (A, h, r, c, X), Y in zip(items, Ymix)])
    b.run()
    order = list(range(len(items)))[::-1]
    Yrev = [torch.empty((y.shape[0], y.stride(0)), dtype=y.dtype, device="cuda")[:, :y.shape[1]] for y in Ymix]
    b.set([(items[i][1], items[i][4], Yrev[i], False) for i in order])  # same items, another order
    b.run()
    for i, (A, h, r, c, X) in enumerate(items):
        Yalone = torch.empty((A.rows, X.stride(0)), dtype=X.dtype, device="cuda")[:, :X.shape[1]]
        b1 = maxe.Batch(1)
        b1.set([(h, X, Yalone, False)])
        b1.run()
        torch.cuda.synchronize()
        assert torch.equal(Yalone, Ymix[i]), i
        assert torch.equal(Yrev[i], Ymix[i]), i


def test_batch_tune_keeps_results():
    A = W.poisson_uniform(3, 50000, 30.0, "f32")
    items = _setup([A, A], [1, 8], seed=3)
    for (A_, h, r, c, X) in items:
        maxe.maxe_batch_tune(h, X.shape[1])
        H, t, it = maxe.maxe_batch_plan_info(h)
        assert H >= 256 and t >= 1 and it in (8, 16)
    b = maxe.Batch(2)
    Ys = [torch.empty((A.rows, X.shape[1]), dtype=X.dtype, device="cuda") for A_, h, r, c, X in items]
    b.set([(h, X, Y, False) for (A_, h, r, c, X), Y in zip(items, Ys)])
    b.run()
    torch.cuda.synchronize()
    for (A_, h, r, c, X), Y in zip(items, Ys):
        _check_against_oracle(A_, r, c, X, Y, False)


@pytest.mark.parametrize("k", [1, 8])
def test_batch_tune_is_never_slower_than_the_default_plan(k):
    """Two handles of one matrix, one with the default batch plan and one tuned:
    a batch of copies of the tuned item takes no longer than the same batch of
    the default item (5% timing margin); the tuned plan keeps the product."""
    A = W.poisson_uniform(4, 120000, 24.0, "f32")
    (A_, hd, r, c, X), = _setup([A], [k], seed=4)
    ht = maxe.from_csr(A_.to("cuda"), r, c)
    maxe.maxe_batch_tune(ht, k)
    assert maxe.maxe_batch_plan_shape(ht) >= 0

    def batch_ms(h, copies=16, reps=5):
        Y = torch.empty((A.rows, X.shape[1]), dtype=X.dtype, device="cuda")
        b = maxe.Batch(copies)
        b.set([(h, X, Y, False)] * copies)
        for _ in range(3):
            b.run()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                b.run()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        b.close()
        return best, Y

    t_def, _ = batch_ms(hd)
    t_tuned, Y = batch_ms(ht)
    assert t_tuned <= 1.05 * t_def, (t_tuned, t_def, maxe.maxe_batch_plan_info(ht))
    _check_against_oracle(A_, r, c, X, Y, False)


def test_batch_run_in_cuda_graph():
    mats = [W.poisson_uniform(60 + i, 20000 + 7000 * i, 12.0, "f32") for i in range(5)]
    items = _setup(mats, [1, 4, 2, 16, 3], seed=11)
    b = maxe.Batch(len(items))
    Ys = [torch.zeros((A.rows, X.shape[1]), dtype=X.dtype, device="cuda") for A, h, r, c, X in items]
    b.set([(h, X, Y, True) for (A, h, r, c, X), Y in zip(items, Ys)])
    b.run()
    torch.cuda.synchronize()
    ref = [y.clone() for y in Ys]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run()
    for y in Ys:
        y.zero_()
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for y, r_ in zip(Ys, ref):
        assert torch.equal(y, r_)


def test_batch_items_without_nonzeros_are_zero():
    """Items with no nonzeros -- no columns at all, or an empty pattern -- come
    out as zeros without any kernel reading their X (which holds no element
    when there are no columns); the other items keep the bits they have alone."""
    mats = [edge_matrix("ragged", "f32", seed=5), W.from_lengths(1, [0] * 7, 0, "f32"),
            W.from_lengths(1, [0] * 9, 13, "f64")]
    ks = [3, 2, 5]
    g = torch.Generator().manual_seed(11)
    items, Ys = [], []
    for A, k in zip(mats, ks):
        vt = torch.float64 if A.dtype == "f64" else torch.float32
        ld = (k + 3) // 4 * 4
        X = torch.rand(A.cols, ld, generator=g, dtype=torch.float64).to(vt).cuda()[:, :k]
        Y = torch.full((A.rows, ld), float("nan"), dtype=vt, device="cuda")[:, :k]
        items.append((maxe.from_csr(A.to("cuda")), X))
        Ys.append(Y)
    b = maxe.Batch(len(items))
    b.set([(h, X, Y, False) for (h, X), Y in zip(items, Ys)])
    b.run()
    h, X = items[0]
    Yalone = torch.full((mats[0].rows, 4), float("nan"), device="cuda")[:, :3]
    b1 = maxe.Batch(1)
    b1.set([(h, X, Yalone, False)])
    b1.run()
    torch.cuda.synchronize()
    assert torch.equal(Ys[0], Yalone)
    assert torch.equal(Ys[1], torch.zeros_like(Ys[1]))
    assert torch.equal(Ys[2], torch.zeros_like(Ys[2]))


def test_batch_rejects_bad_items():
    A = edge_matrix("ragged", "f32")
    h = maxe.from_csr(A.to("cuda"))
    b = maxe.Batch(2)
    X = torch.zeros(A.cols, 65, device="cuda")
    Y = torch.zeros(A.rows, 65, device="cuda")
    with pytest.raises(maxe.MaxeError):
        b.set([(h, X, Y, False)])
    with pytest.raises(maxe.MaxeError):
        b.set([(h, X[:, :2].contiguous(), Y[:, :2].contiguous(), False)] * 3)  # over capacity
