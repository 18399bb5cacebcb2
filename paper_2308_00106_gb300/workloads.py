"""Seeded synthetic sparse matrices and vectors shaped like the paper's workloads.

This module only makes inputs. It holds none of the method's arithmetic (no
permutation, no entropy, no product), and both the CUDA path and the CPU oracle
consume what it makes. Generation uses torch random streams on the requested
device: the same seed gives the same matrix on the same kind of device, so a
test makes its input once and hands copies to both sides.

The paper measured public sparse matrices (OPF 3754, LP OSA 07, MULT DCOP 01/03,
Section 6). They are not available here; these generators stand in for them:

  blockdiag      4096 x 4096, 16 diagonal 256 x 256 blocks with each entry
                 present with probability 0.02, plus 2000 distinct uniform
                 off-block entries; FP64 values U[-1, 1].
  powerlaw       2^20 x 2^20; row lengths Zipf(1.5) restricted to 1..1000
                 (rejection sampling of Zipf above the cap is the same as
                 drawing from the truncated law); columns i + round(N(0, 2000)),
                 redrawn when outside the matrix or already used in the row;
                 FP32 values U[-1, 1].
  laplacian5     5-point stencil on an n x n grid (diagonal 4, neighbours -1,
                 Dirichlet: missing neighbours dropped), natural row order.
  poisson_uniform  square, Poisson(lam) row lengths, distinct uniform columns.
  batched_set / serving_set  the lists of matrices of the batched and served forms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

DTYPES = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
DTYPE_CODE = {"f64": 0, "f32": 1, "bf16": 2}


@dataclass
class CSR:
    """CSR with int32 row pointers and columns, ascending columns in each row."""

    rows: int
    cols: int
    rowptr: torch.Tensor  # int32 [rows + 1]
    col: torch.Tensor  # int32 [nnz]
    val: torch.Tensor  # float64 / float32 / bfloat16 [nnz]
    dtype: str  # "f64" | "f32" | "bf16"

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def device(self) -> torch.device:
        return self.col.device

    def to(self, device) -> "CSR":
        return CSR(self.rows, self.cols, self.rowptr.to(device), self.col.to(device), self.val.to(device), self.dtype)

    def astype(self, dtype: str) -> "CSR":
        return CSR(self.rows, self.cols, self.rowptr, self.col, self.val.to(DTYPES[dtype]), dtype)

    def numpy(self):
        """(rowptr int32, col int32, val) with bf16 values as their uint16 bit patterns."""
        v = self.val.cpu()
        if self.dtype == "bf16":
            v = v.view(torch.int16).numpy().view(np.uint16)
        else:
            v = v.numpy()
        return self.rowptr.cpu().numpy(), self.col.cpu().numpy(), v


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _uniform(n: int, g: torch.Generator, device, dtype: str) -> torch.Tensor:
    u = torch.rand(n, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0
    return u.to(DTYPES[dtype])


def vector(seed: int, n: int, dtype: str = "f64", device="cpu") -> torch.Tensor:
    """U[-1, 1] entries (float64 or float32)."""
    return _uniform(n, _gen(seed, device), device, dtype)


def matrix_rhs(seed: int, n: int, k: int, dtype: str = "f32", device="cpu") -> torch.Tensor:
    """Row-major n x k block of right-hand sides, U[-1, 1]."""
    return _uniform(n * k, _gen(seed, device), device, dtype).reshape(n, k)


def _from_sorted_keys(keys: torch.Tensor, rows: int, cols: int, val: torch.Tensor, dtype: str) -> CSR:
    r = torch.div(keys, cols, rounding_mode="floor")
    c = (keys - r * cols).to(torch.int32)
    counts = torch.bincount(r, minlength=rows)
    rowptr = torch.zeros(rows + 1, dtype=torch.int64, device=keys.device)
    rowptr[1:] = torch.cumsum(counts, 0)
    return CSR(rows, cols, rowptr.to(torch.int32), c.contiguous(), val.contiguous(), dtype)


def _distinct_columns(row_of: torch.Tensor, draw, rows: int, cols: int, g, device, max_rounds: int = 200):
    """Draw a column for every entry with draw(idx) and redraw entries that fall
    outside [0, cols) or repeat a column already used in their row. Returns the
    sorted row-major keys row * cols + col."""
    n = row_of.numel()
    colv = torch.empty(n, dtype=torch.int64, device=device)
    need = torch.arange(n, device=device)
    for _ in range(max_rounds):
        if need.numel() == 0:
            break
        colv[need] = draw(need)
        bad = need[(colv[need] < 0) | (colv[need] >= cols)]
        colv[bad] = -1
        valid = colv >= 0
        keys = torch.where(valid, row_of * cols + colv, torch.full_like(colv, -1))
        sk, order = torch.sort(keys, stable=True)
        dup = torch.zeros(n, dtype=torch.bool, device=device)
        if n > 1:
            dup[1:] = (sk[1:] == sk[:-1]) & (sk[1:] >= 0)
        dup_idx = order[dup]
        need = torch.cat([bad, dup_idx])
    else:
        raise RuntimeError("could not draw distinct columns")
    keys = row_of * cols + colv
    return torch.sort(keys).values


def from_lengths(seed: int, lengths, cols: int, dtype: str = "f32", device="cpu") -> CSR:
    """Rows of the given lengths with distinct uniform columns and U[-1,1] values."""
    lengths = torch.as_tensor(lengths, dtype=torch.int64, device=device)
    rows = lengths.numel()
    if int(lengths.max().item() if rows else 0) > cols:
        raise ValueError("row longer than the number of columns")
    g = _gen(seed, device)
    row_of = torch.repeat_interleave(torch.arange(rows, device=device), lengths)
    n = row_of.numel()
    if n == 0:
        return CSR(rows, cols, torch.zeros(rows + 1, dtype=torch.int32, device=device),
                   torch.zeros(0, dtype=torch.int32, device=device), torch.zeros(0, dtype=DTYPES[dtype], device=device),
                   dtype)
    # dense rows: draw a random subset directly to avoid endless redraws
    keys = _distinct_columns(row_of, lambda idx: torch.randint(0, cols, (idx.numel(),), generator=g, device=device),
                             rows, cols, g, device, max_rounds=10000)
    val = _uniform(n, g, device, dtype)
    return _from_sorted_keys(keys, rows, cols, val, dtype)


def blockdiag(seed: int = 2308, n: int = 4096, blocks: int = 16, fill: float = 0.02, offblock: int = 2000,
              dtype: str = "f64", device="cpu") -> CSR:
    """4096 x 4096: 16 dense-ish diagonal blocks at 2% fill plus 2000 uniform off-block entries."""
    g = _gen(seed, device)
    bs = n // blocks
    mask = torch.rand((blocks, bs, bs), generator=g, device=device) < fill
    b, r, c = torch.nonzero(mask, as_tuple=True)
    keys_in = (b * bs + r) * n + (b * bs + c)
    # distinct off-block entries
    chosen = torch.empty(0, dtype=torch.int64, device=device)
    while chosen.numel() < offblock:
        m = 2 * (offblock - chosen.numel()) + 16
        i = torch.randint(0, n, (m,), generator=g, device=device)
        j = torch.randint(0, n, (m,), generator=g, device=device)
        ok = (i // bs) != (j // bs)
        cand = (i * n + j)[ok]
        for kk in cand.tolist():
            if chosen.numel() >= offblock:
                break
            if not bool((chosen == kk).any()):
                chosen = torch.cat([chosen, torch.tensor([kk], device=device)])
    keys = torch.sort(torch.cat([keys_in, chosen])).values
    val = _uniform(keys.numel(), g, device, dtype)
    return _from_sorted_keys(keys, n, n, val, dtype)


def zipf_lengths(n: int, s: float, cap: int, g, device) -> torch.Tensor:
    """Row lengths from Zipf(s) restricted to 1..cap (inverse CDF of the truncated law)."""
    k = torch.arange(1, cap + 1, dtype=torch.float64, device=device)
    pmf = k.pow(-s)
    cdf = torch.cumsum(pmf, 0)
    cdf = cdf / cdf[-1]
    u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    idx = torch.searchsorted(cdf, u, right=True).clamp_(max=cap - 1)
    return idx + 1


def powerlaw(seed: int = 2308, n: int = 1 << 20, zipf_s: float = 1.5, cap: int = 1000, sigma: float = 2000.0,
             dtype: str = "f32", device="cpu", length_scale: float = 1.0) -> CSR:
    """Power-law row lengths, columns clustered near the diagonal (Gaussian)."""
    g = _gen(seed, device)
    lengths = zipf_lengths(n, zipf_s, cap, g, device)
    if length_scale != 1.0:
        lengths = torch.clamp((lengths.double() * length_scale).round().long(), min=1)
    row_of = torch.repeat_interleave(torch.arange(n, device=device), lengths)

    def draw(idx):
        off = torch.round(torch.randn(idx.numel(), generator=g, device=device, dtype=torch.float64) * sigma)
        return row_of[idx] + off.long()

    keys = _distinct_columns(row_of, draw, n, n, g, device)
    val = _uniform(keys.numel(), g, device, dtype)
    return _from_sorted_keys(keys, n, n, val, dtype)


def laplacian5(n: int = 4096, dtype: str = "f64", device="cpu") -> CSR:
    """5-point Laplacian on an n x n grid, natural (row-major) order."""
    M = n * n
    idx = torch.arange(M, device=device, dtype=torch.int64)
    p, q = idx // n, idx % n
    cols = torch.stack([idx - n, idx - 1, idx, idx + 1, idx + n], 1)
    present = torch.stack([p > 0, q > 0, torch.ones_like(p, dtype=torch.bool), q < n - 1, p < n - 1], 1)
    vals = torch.tensor([-1.0, -1.0, 4.0, -1.0, -1.0], dtype=torch.float64, device=device).expand(M, 5)
    counts = present.sum(1)
    rowptr = torch.zeros(M + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(counts, 0)
    col = cols[present].to(torch.int32)
    val = vals[present].to(DTYPES[dtype])
    return CSR(M, M, rowptr.to(torch.int32), col.contiguous(), val.contiguous(), dtype)


def poisson_uniform(seed: int, rows: int, lam: float, dtype: str = "f32", device="cpu", cols: int | None = None) -> CSR:
    """Square (unless cols given) matrix with Poisson(lam) row lengths and distinct uniform columns."""
    cols = rows if cols is None else cols
    g = _gen(seed, device)
    lengths = torch.poisson(torch.full((rows,), float(lam), dtype=torch.float64, device=device), generator=g)
    lengths = lengths.long().clamp_(max=cols)
    return from_lengths(seed ^ 0x5DEECE66D, lengths, cols, dtype, device)


def batched_set(seed: int = 2308, count: int = 256, rows_lo: int = 1000, rows_hi: int = 200_000,
                lam_lo: float = 8.0, lam_hi: float = 64.0, kmax: int = 16, dtype: str = "f32", device="cpu"):
    """Uneven matrices (rows log-uniform, Poisson row lengths), each with 1..kmax right-hand sides."""
    rng = np.random.default_rng(seed)
    rows = np.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi), count)).round().astype(np.int64)
    lams = rng.uniform(lam_lo, lam_hi, count)
    ks = rng.integers(1, kmax + 1, count)
    mats = [poisson_uniform(seed * 1000 + m, int(rows[m]), float(lams[m]), dtype, device) for m in range(count)]
    return mats, [int(k) for k in ks]


def serving_set(seed: int = 2308, count: int = 64, rows_lo: int = 10_000, rows_hi: int = 4_000_000,
                lam_lo: float = 5.0, lam_hi: float = 50.0, device="cpu"):
    """Resident matrices of the serving loop, half FP32 and half BF16 values."""
    rng = np.random.default_rng(seed + 1)
    rows = np.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi), count)).round().astype(np.int64)
    lams = rng.uniform(lam_lo, lam_hi, count)
    return [poisson_uniform(seed * 7919 + m, int(rows[m]), float(lams[m]), "f32" if m % 2 == 0 else "bf16", device)
            for m in range(count)]


def clustered_heavy(seed: int = 2308, n: int = 1 << 20, heavy_frac: float = 0.01, heavy_len: int = 1000,
                    light_len: int = 16, dtype: str = "f32", device="cpu") -> CSR:
    """Rows of two lengths, the heavy ones contiguous at the top: the shape Section 5
    reports for LP OSA 07 (a handful of long rows next to one another), under which a
    fixed equal-rows split is unbalanced until the rows are permuted. Distinct
    uniform columns, U[-1, 1] values."""
    nh = int(round(n * heavy_frac))
    lengths = torch.full((n,), light_len, dtype=torch.int64, device=device)
    lengths[:nh] = heavy_len
    return from_lengths(seed, lengths, n, dtype, device)
