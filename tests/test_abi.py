"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/*.h declares (no compute calls: this file runs on CPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2308_00106_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^MAXE_API\s+[\w\s\*]+?\b(maxe_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["maxe_build_permutation", "maxe_permute_csr", "maxe_nnz_entropy", "maxe_spmv", "maxe_spmm",
                 "maxe_handle_destroy", "maxe_status_str"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (maxe_\w+)", out))
    assert exported == set(declared_symbols()), exported ^ set(declared_symbols())


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.maxe_status_str.restype = ctypes.c_char_p
    lib.maxe_status_str.argtypes = [ctypes.c_int]
    assert lib.maxe_status_str(0) == b"MAXE_OK"
    assert lib.maxe_status_str(4) == b"MAXE_ERR_TIMEOUT"
    lib.maxe_version.restype = ctypes.c_char_p
    assert re.match(rb"\d+\.\d+\.\d+", lib.maxe_version())


def test_host_checks_reject_bad_arguments_without_launching(lib_path):
    """Argument checks run on the host before any CUDA call."""
    lib = ctypes.CDLL(lib_path)
    lib.maxe_build_permutation.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
    assert lib.maxe_build_permutation(1, -5, 0, None, None, None) == 1
    assert lib.maxe_build_permutation(1, 5, 7, None, None, None) == 1
    assert lib.maxe_build_permutation(1, 0, 0, None, None, None) == 0
    lib.maxe_spmv.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_uint32, ctypes.c_void_p]
    assert lib.maxe_spmv(None, None, None, 0, None) == 1
    lib.maxe_spmv_host.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_uint32, ctypes.c_void_p]
    assert lib.maxe_spmv_host(None, None, None, None, None, 0, None) == 1
    assert lib.maxe_spmv_host(None, None, None, None, None, 0x80, None) == 1
    lib.maxe_handle_destroy.argtypes = [ctypes.c_void_p]
    assert lib.maxe_handle_destroy(None) == 0


def test_build_uses_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
