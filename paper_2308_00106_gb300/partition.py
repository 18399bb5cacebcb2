"""Row blocks of a permuted matrix over ranks (one GPU per rank).

The paper's laggard argument (Section 3, randomization): with a random row
permutation, blocks of equal row counts carry nearly equal numbers of
nonzeros, so no rank waits for a slow one.  Here the blocks are cut at equal
nonzero counts directly (the first row whose start reaches k * nnz / p), which
balances the product whatever the order of the rows.

Each rank owns the rows [r_k, r_{k+1}) of A' and computes its slice of
y' = A' x' -- disjoint rows, no reduction.  Iterative use (the power iteration
of the serving loop, any Krylov method) needs the whole vector on every rank
for the next product: an all-gather of the slices, the one exchange step.

The per-rank product is a callable: on a GPU, `gpu_block_product` builds a
library handle from the block (its own nnz-balanced warp partition, x-sliced
form when it pays) and runs maxe_spmv; the tests run the host logic on CPU
ranks with a reference product instead.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


def row_blocks(rowptr, parts: int) -> np.ndarray:
    """Split points r_0 = 0 <= r_1 <= ... <= r_p = rows: block k holds the rows
    whose first entry lies in [k * nnz / p, (k + 1) * nnz / p) (by rows' starts,
    so a row is never split); the last block also takes trailing empty rows."""
    rp = np.asarray(rowptr, dtype=np.int64)
    rows = len(rp) - 1
    if parts < 1:
        raise ValueError("parts must be >= 1")
    nnz = int(rp[-1])
    cuts = np.empty(parts + 1, dtype=np.int64)
    cuts[0], cuts[parts] = 0, rows
    for k in range(1, parts):
        target = (k * nnz + parts - 1) // parts
        cuts[k] = int(np.searchsorted(rp[:rows], target, side="left"))
    return np.maximum.accumulate(cuts)


@dataclass
class Block:
    """Rows [r0, r1) of a CSR matrix: rowptr rebased to 0, columns and values sliced."""
    r0: int
    r1: int
    cols: int
    rowptr: object
    col: object
    val: object
    handle: object = None  # the library handle of the block, made on first use on a GPU

    @property
    def rows(self) -> int:
        return self.r1 - self.r0

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def block_of(rowptr, col, val, cols: int, r0: int, r1: int) -> Block:
    """The CSR rows [r0, r1) (numpy arrays or torch tensors on any device)."""
    e0, e1 = int(rowptr[r0]), int(rowptr[r1])
    rp = rowptr[r0:r1 + 1] - e0
    return Block(int(r0), int(r1), int(cols), rp, col[e0:e1], val[e0:e1])


class RowBlockProduct:
    """y' = A' x' over `world` ranks: rank `rank` multiplies its row block with
    `local_product(block, x) -> y_block` and the slices are all-gathered, so
    every rank ends with the whole y' (rows in order)."""

    def __init__(self, rowptr, col, val, cols: int, rank: int, world: int, local_product, group=None):
        rp_host = rowptr.cpu().numpy() if isinstance(rowptr, torch.Tensor) else np.asarray(rowptr)
        self.cuts = row_blocks(rp_host, world)
        self.rank, self.world, self.group = rank, world, group
        self.rows = len(rp_host) - 1
        r0, r1 = int(self.cuts[rank]), int(self.cuts[rank + 1])
        self.block = block_of(rowptr, col, val, cols, r0, r1)
        self.local_product = local_product
        self.max_rows = int(np.max(np.diff(self.cuts)))
        # nonzeros of every rank's block: the balance the partition gives
        self.block_nnz = [int(rp_host[self.cuts[k + 1]] - rp_host[self.cuts[k]]) for k in range(world)]

    def step(self, x: torch.Tensor) -> torch.Tensor:
        """The whole y' = A' x' on every rank (x' whole on every rank)."""
        y_blk = self.local_product(self.block, x)
        if self.world == 1:
            return y_blk
        import torch.distributed as dist
        pad = torch.zeros(self.max_rows, dtype=y_blk.dtype, device=y_blk.device)
        pad[:y_blk.numel()] = y_blk
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        return torch.cat([parts[k][:int(self.cuts[k + 1] - self.cuts[k])] for k in range(self.world)])


def gpu_block_product(autotune: bool = True):
    """A local product for RowBlockProduct on this rank's GPU: a library handle
    of the block (built once, on first use) and maxe_spmv with vectors in the
    permuted space."""
    from . import maxe
    from .workloads import CSR

    def product(block: Block, x: torch.Tensor) -> torch.Tensor:
        if block.handle is None:
            dtype = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}[block.val.dtype]
            A = CSR(block.rows, block.cols, block.rowptr.to(torch.int32), block.col, block.val, dtype)
            block.handle = maxe.from_csr(A, autotune=autotune)
        return maxe.maxe_spmv(block.handle, x, permuted=True)

    return product
