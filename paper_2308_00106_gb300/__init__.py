"""max_E SpMV for GB300: entropy-maximising random permutation of a sparse
matrix plus CSR SpMV/SpMM on the permuted matrix (arXiv 2308.00106, Eq. 1).

The compute path is the C-ABI CUDA library ``libmaxe.so`` (sources in
``csrc/``, declarations in ``include/maxe.h``); ``maxe`` is its thin ctypes
binding and ``workloads`` makes the seeded synthetic inputs. Importing the
package itself loads nothing.
"""
__all__ = ["maxe", "workloads"]
