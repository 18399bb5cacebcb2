"""The row-block partition over ranks, on CPU: blocks of equal nonzeros (each
within one row of nnz / p), and two `gloo` ranks that multiply their blocks of
a permuted power-law matrix and all-gather the slices get the whole product,
equal bit for bit to the oracle's product of the whole matrix (each row is
summed by the same code in the same order), and again after a second step
fed with the first step's result (the iterative use)."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_00106_gb300 import partition  # noqa: E402
from paper_2308_00106_gb300 import workloads as W  # noqa: E402


def _matrix():
    A = W.powerlaw(17, n=30000, device="cpu")
    rp, co, va = A.numpy()
    r = oracle.build_permutation(17, A.rows, 0)
    c = oracle.build_permutation(17, A.cols, 1)
    prp, pco, pva = oracle.permute_csr(A.rows, A.cols, rp, co, va, W.DTYPE_CODE["f32"], r, c)
    return A.rows, A.cols, prp, pco, pva


@pytest.mark.parametrize("parts", [1, 2, 3, 7, 64])
def test_row_blocks_have_equal_nonzeros(parts):
    M, N, rp, co, va = _matrix()
    cuts = partition.row_blocks(rp, parts)
    assert cuts[0] == 0 and cuts[-1] == M and (np.diff(cuts) >= 0).all()
    nnz = np.diff(rp[cuts])
    longest = int(np.diff(rp).max())
    assert nnz.sum() == rp[-1]
    assert (np.abs(nnz - rp[-1] / parts) <= longest + 1).all()


def test_row_blocks_degenerate_cases():
    assert list(partition.row_blocks(np.array([0]), 3)) == [0, 0, 0, 0]  # no rows
    assert list(partition.row_blocks(np.array([0, 0, 0]), 2)) == [0, 0, 2]  # no entries: all to the last block
    assert list(partition.row_blocks(np.array([0, 5]), 4)) == [0, 1, 1, 1, 1]  # one row: one block takes it
    with pytest.raises(ValueError):
        partition.row_blocks(np.array([0, 1]), 0)


def _oracle_product(block, x):
    y = oracle.spmv(block.rows, block.rowptr, block.col, block.val, W.DTYPE_CODE["f32"], x.numpy())
    return torch.from_numpy(y)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M, N, rp, co, va = _matrix()
        pr = partition.RowBlockProduct(rp, co, va, N, rank, world, _oracle_product)
        x = torch.from_numpy(W.vector(5, N, "f64", "cpu").numpy())
        y1 = pr.step(x)
        x2 = y1.numpy() / np.linalg.norm(y1.numpy())  # the same normalisation as the reference's
        y2 = pr.step(torch.from_numpy(x2))
        np.save(os.path.join(out_dir, f"y1_{rank}.npy"), y1.numpy())
        np.save(os.path.join(out_dir, f"y2_{rank}.npy"), y2.numpy())
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"block_nnz": pr.block_nnz, "rows": [int(pr.cuts[rank]), int(pr.cuts[rank + 1])]}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_whole_product(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    M, N, rp, co, va = _matrix()
    x = W.vector(5, N, "f64", "cpu").numpy()
    ref1 = oracle.spmv(M, rp, co, va, W.DTYPE_CODE["f32"], x)
    ref2 = oracle.spmv(M, rp, co, va, W.DTYPE_CODE["f32"], ref1 / np.linalg.norm(ref1))
    meta = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert meta[0]["rows"][1] == meta[1]["rows"][0]  # adjacent, disjoint row blocks
    assert sum(meta[0]["block_nnz"]) == rp[-1]
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"y1_{r}.npy"), ref1)
        np.testing.assert_array_equal(np.load(tmp_path / f"y2_{r}.npy"), ref2)
