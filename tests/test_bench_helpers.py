"""The benchmark's bookkeeping, on CPU: algorithmic bytes, the ncu traffic
records it quotes (tied to the hash of the kernel's sources), the host record
of CPU numbers."""
import json
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


def _fake_ncu_csv(path, kernel_name, read_mb, write_mb):
    hdr = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"]
    units = ["", "", "Mbyte", "Mbyte", "nsecond"]
    rows = [hdr, units, ["0", kernel_name, f"{read_mb:,.3f}", f"{write_mb:,.3f}", "85,000"],
            ["1", "other_kernel", "1", "1", "1"]]
    with open(path, "w") as f:
        for r in rows:
            f.write(",".join(f'"{c}"' for c in r) + "\n")


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_SOURCES))
def test_traffic_records_are_tied_to_the_kernel_sources(kernel, tmp_path):
    csv = tmp_path / "raw.csv"
    _fake_ncu_csv(csv, f"void maxe::{kernel}<float, float, 2, false>(Params)", 1227.5, 3.1)
    rec = bench.record_profile(str(csv), kernel, 0, "ncu ...", "powerlaw", out_dir=str(tmp_path))
    assert rec["traffic_bytes_per_launch"] == pytest.approx(1230.6e6)
    assert rec["source_sha256"] == bench.kernel_source_hash(kernel)
    assert bench.traffic_from_record(kernel, str(tmp_path)) == pytest.approx(1230.6e6)
    # a record taken on other sources is not quoted
    rec["source_sha256"] = "0" * 64
    (tmp_path / bench.PROFILE_RECORD[kernel]).write_text(json.dumps(rec))
    assert bench.traffic_from_record(kernel, str(tmp_path)) is None


def test_host_record():
    h = bench.host_info()
    assert h["nproc"] >= 1 and h["machine"]


def test_headline_kernel_record_matches_its_sources():
    # The roofline's traffic for the headline kernel comes from this record; a
    # change to the kernel's sources must come with a new ncu capture.
    p = os.path.join(ROOT, "profiles", bench.PROFILE_RECORD["spmv_xslice_kernel"])
    assert os.path.exists(p), "no ncu record of spmv_xslice_kernel under profiles/"
    rec = json.load(open(p))
    assert rec["source_sha256"] == bench.kernel_source_hash("spmv_xslice_kernel"), \
        "xslice.cu or internal.cuh changed since the ncu record was taken: capture and record it again"
    alg = bench.alg_bytes(1 << 20, 1 << 20, 25394653, 4, 4, 4)
    assert 0.9 * alg < rec["traffic_bytes_per_launch"] < 3 * alg


def test_bench_rejects_an_empty_e2e_stream_rotation():
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--e2e-streams", "0"],
                       capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 2
    assert "--e2e-streams must be at least 1" in r.stderr
