"""The per-rank product of the row-block partition on a GPU: three blocks of a
permuted power-law matrix, each a library handle of its own (rebased row
pointers), multiplied one after another on one GPU; the slices, in order,
give every row of the oracle's product within the FP32 tolerance.  (Several
ranks exchange the slices with an all-gather, tested on CPU ranks.)"""
import pytest
import torch

from paper_2308_00106_gb300 import maxe, partition
from paper_2308_00106_gb300 import workloads as W
from tests.gpu_common import check_all_rows, handle_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    maxe.load(build_if_missing=True)


@pytest.mark.parametrize("parts", [1, 3])
def test_gpu_block_products_concatenate_to_the_whole_product(parts):
    A = W.powerlaw(19, n=200000, device="cuda")
    r = maxe.maxe_build_permutation(19, A.rows, 0)
    c = maxe.maxe_build_permutation(19, A.cols, 1)
    h = maxe.from_csr(A, r, c)
    rp, co, va, _, _ = h.csr()  # the permuted CSR A'
    cuts = partition.row_blocks(rp.cpu().numpy(), parts)
    product = partition.gpu_block_product(autotune=True)
    x = W.vector(3, A.cols, "f32", "cuda")
    ys = []
    for k in range(parts):
        blk = partition.block_of(rp, co, va, A.cols, int(cuts[k]), int(cuts[k + 1]))
        ys.append(product(blk, x))
    y = torch.cat(ys)
    nrp, nco, nva = handle_arrays(h)
    check_all_rows(y.cpu().numpy(), nrp, nco, nva, "f32", x.cpu().numpy())
