"""A plain C99 program (tests/c/abi_laplacian.c) compiles against include/maxe.h
with strict warnings and links against libmaxe.so (CPU), and on a GPU runs the
whole path -- permutations, permuted CSR, entropy, SpMV -- through the C-ABI
alone, checked against the 1-D Laplacian's closed form."""
import glob
import os
import shutil
import subprocess

import pytest

from paper_2308_00106_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_laplacian.c")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _cudart_dir(home):
    for cand in [os.path.join(home, "lib64")] + sorted(glob.glob(os.path.join(home, "targets", "*", "lib"))):
        if glob.glob(os.path.join(cand, "libcudart.so*")):
            return cand
    pytest.skip("libcudart.so not found")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = B.build()
    libdir = os.path.dirname(lib)
    home = _cuda_home()
    exe = str(tmp_path_factory.mktemp("cabi") / "abi_laplacian")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(home, "include"),
           SRC, "-o", exe, "-L", libdir, "-lmaxe", "-Wl,-rpath," + libdir,
           "-L", _cudart_dir(home), "-lcudart", "-Wl,-rpath," + _cudart_dir(home)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_compiles_and_links(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("n,seed", [(3, 1), (4099, 2), (100003, 7)])
def test_c_client_runs_the_path(client, n, seed):
    r = subprocess.run([client, str(n), str(seed)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 wrong" in r.stdout
