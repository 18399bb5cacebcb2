"""Shape checks of the seeded synthetic inputs (CPU)."""
import numpy as np
import pytest
import torch

from paper_2308_00106_gb300 import workloads as W


def _valid_csr(A):
    rp, co, _ = A.numpy()
    assert rp[0] == 0 and rp[-1] == A.nnz and np.all(np.diff(rp) >= 0)
    assert A.nnz == 0 or (co.min() >= 0 and co.max() < A.cols)
    for i in range(A.rows):
        seg = co[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_laplacian_counts():
    A = W.laplacian5(64, "bf16")
    assert A.rows == 4096 and A.nnz == 5 * 64 * 64 - 4 * 64
    _valid_csr(A)


def test_blockdiag_structure():
    A = W.blockdiag(2308, n=1024, blocks=4, fill=0.02, offblock=200)
    _valid_csr(A)
    rp, co, _ = A.numpy()
    rows = np.repeat(np.arange(A.rows), np.diff(rp))
    off = (rows // 256) != (co // 256)
    assert off.sum() == 200
    assert A.val.dtype == torch.float64 and float(A.val.abs().max()) <= 1.0


def test_powerlaw_small():
    A = W.powerlaw(1, n=20000, cap=300, sigma=200.0)
    _valid_csr(A)
    lengths = np.diff(A.numpy()[0])
    assert lengths.min() >= 1 and lengths.max() <= 300
    # truncated Zipf(1.5): P(len = 1) = 1 / sum_{k<=300} k^-1.5
    p1 = 1.0 / np.sum(np.arange(1, 301, dtype=np.float64) ** -1.5)
    assert abs((lengths == 1).mean() - p1) < 0.02
    rp, co, _ = A.numpy()
    rows = np.repeat(np.arange(A.rows), lengths)
    assert np.abs(co - rows).std() < 400


def test_from_lengths_edge_cases():
    A = W.from_lengths(3, [0, 0, 5, 0, 1, 7], 7, "f64")
    _valid_csr(A)
    assert np.array_equal(np.diff(A.numpy()[0]), [0, 0, 5, 0, 1, 7])
    E = W.from_lengths(3, [0, 0, 0], 4, "f32")
    assert E.nnz == 0


def test_poisson_uniform_and_reproducible():
    A = W.poisson_uniform(9, 3000, 12.0)
    B = W.poisson_uniform(9, 3000, 12.0)
    _valid_csr(A)
    assert torch.equal(A.col, B.col) and torch.equal(A.val, B.val)
    assert abs(A.nnz / 3000 - 12.0) < 0.5
