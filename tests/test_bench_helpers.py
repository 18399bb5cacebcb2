"""The benchmark's bookkeeping, on CPU: algorithmic bytes, the committed ncu
traffic it quotes (and the kernel revision those counters belong to), the
host record of CPU numbers."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_count_every_byte_once():
    # nnz (value + index) + (M + 1) row pointers + M*k outputs + N*k inputs
    assert bench.alg_bytes(10, 20, 100, 4, 4, 4) == 100 * 8 + 11 * 4 + 10 * 4 + 20 * 4
    assert bench.alg_bytes(10, 20, 100, 2, 4, 4, k=3) == 100 * 6 + 11 * 4 + 10 * 3 * 4 + 20 * 3 * 4
    # the 1M-row power-law FP32 product quoted in the profiles
    assert bench.alg_bytes(1 << 20, 1 << 20, 25394653, 4, 4, 4) == 215740140


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_REVISION))
def test_profiles_match_the_kernel_revisions_the_bench_quotes(kernel):
    traffic, rev = bench.traffic_from_profile(bench.PROFILE_OF[kernel])
    assert rev == bench.KERNEL_REVISION[kernel], "profile taken on another revision of the kernel"
    # DRAM bytes per launch near the algorithmic bytes of the profiled product
    assert 0.95 * 215740140 <= traffic <= 1.1 * 215740140


def test_host_record():
    h = bench.host_info()
    assert h["nproc"] >= 1 and h["machine"]
