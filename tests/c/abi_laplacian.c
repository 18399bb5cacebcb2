/* A plain C99 client of the C-ABI: no Python, no PyTorch.  It builds the 1-D
 * Laplacian (tridiagonal 2, -1, -1) of order n on the host, copies it to the
 * device with the CUDA runtime, draws both permutations (Section 3), permutes
 * the matrix (Eq. 1), runs y = A x through the permuted handle and checks the
 * closed form for x_i = i: every interior row sums to 2i - (i-1) - (i+1) = 0,
 * the first row gives -1 and the last 2(n-1) - (n-2) = n.  All values are
 * small integers, so FP64 results are exact whatever the summation order.
 * It also checks the entropy of a 1 x 1 grid (0) and that an unknown flag is
 * refused on the host.  Exit status 0 on success, 1 on a wrong result, 2 on an
 * error status from the library or the runtime. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "maxe.h"

#define CHECK_CUDA(call)                                                   \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return 2;                                                            \
    }                                                                      \
  } while (0)

#define CHECK_MAXE(call)                                                   \
  do {                                                                     \
    maxe_status s_ = (call);                                               \
    if (s_ != MAXE_OK) {                                                   \
      fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, maxe_status_str(s_)); \
      return 2;                                                            \
    }                                                                      \
  } while (0)

int main(int argc, char** argv) {
  int32_t n = argc > 1 ? (int32_t)atoi(argv[1]) : 100003;
  uint64_t seed = argc > 2 ? (uint64_t)strtoull(argv[2], NULL, 10) : 7u;
  if (n < 3) return 2;
  int64_t nnz = 3 * (int64_t)n - 2;

  int32_t* rowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnz);
  double* val = (double*)malloc(sizeof(double) * (size_t)nnz);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!rowptr || !col || !val || !x || !y) return 2;
  int64_t e = 0;
  for (int32_t i = 0; i < n; ++i) {
    rowptr[i] = (int32_t)e;
    if (i > 0) { col[e] = i - 1; val[e++] = -1.0; }
    col[e] = i; val[e++] = 2.0;
    if (i + 1 < n) { col[e] = i + 1; val[e++] = -1.0; }
    x[i] = (double)i;
  }
  rowptr[n] = (int32_t)e;
  if (e != nnz) return 2;

  int32_t *d_rowptr, *d_col, *d_rperm, *d_cperm;
  double *d_val, *d_x, *d_y;
  CHECK_CUDA(cudaMalloc((void**)&d_rowptr, sizeof(int32_t) * (size_t)(n + 1)));
  CHECK_CUDA(cudaMalloc((void**)&d_col, sizeof(int32_t) * (size_t)nnz));
  CHECK_CUDA(cudaMalloc((void**)&d_val, sizeof(double) * (size_t)nnz));
  CHECK_CUDA(cudaMalloc((void**)&d_rperm, sizeof(int32_t) * (size_t)n));
  CHECK_CUDA(cudaMalloc((void**)&d_cperm, sizeof(int32_t) * (size_t)n));
  CHECK_CUDA(cudaMalloc((void**)&d_x, sizeof(double) * (size_t)n));
  CHECK_CUDA(cudaMalloc((void**)&d_y, sizeof(double) * (size_t)n));
  CHECK_CUDA(cudaMemcpy(d_rowptr, rowptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(d_x, x, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));

  maxe_csr A;
  A.rows = n;
  A.cols = n;
  A.nnz = nnz;
  A.rowptr = d_rowptr;
  A.col = d_col;
  A.val = d_val;
  A.dtype = MAXE_F64;

  CHECK_MAXE(maxe_build_permutation(seed, n, 0, d_rperm, NULL, NULL));
  CHECK_MAXE(maxe_build_permutation(seed, n, 1, d_cperm, NULL, NULL));
  maxe_handle* h = NULL;
  CHECK_MAXE(maxe_permute_csr(&A, d_rperm, d_cperm, MAXE_VALIDATE | MAXE_AUTOTUNE, NULL, NULL, &h));

  double H = -1.0;
  CHECK_MAXE(maxe_nnz_entropy(h, 1, 1, 2.0, &H, NULL, NULL, NULL));

  CHECK_CUDA(cudaMemset(d_y, 0xff, sizeof(double) * (size_t)n));
  CHECK_MAXE(maxe_spmv(h, d_x, d_y, 0u, NULL));
  CHECK_MAXE(maxe_device_status(NULL));
  CHECK_CUDA(cudaMemcpy(y, d_y, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));

  maxe_status refused = maxe_spmv(h, d_x, d_y, 0x80000000u, NULL);

  /* the same product from host memory in one call (pageable buffers) */
  double* y2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* d_x2 = NULL;
  if (!y2) return 2;
  CHECK_CUDA(cudaMalloc((void**)&d_x2, sizeof(double) * (size_t)n));
  CHECK_MAXE(maxe_spmv_host(h, x, y2, d_x2, d_y, 0u, NULL));
  CHECK_CUDA(cudaDeviceSynchronize());

  int bad = 0;
  for (int32_t i = 0; i < n; ++i) {
    double want = i == 0 ? -1.0 : (i == n - 1 ? (double)n : 0.0);
    if (y[i] != want) {
      if (bad < 5) fprintf(stderr, "y[%d] = %.17g, want %.17g\n", i, y[i], want);
      ++bad;
    }
  }
  for (int32_t i = 0; i < n; ++i) {
    if (memcmp(&y2[i], &y[i], sizeof(double)) != 0) {
      if (bad < 5) fprintf(stderr, "host-buffer y[%d] = %.17g, device call %.17g\n", i, y2[i], y[i]);
      ++bad;
    }
  }
  if (H != 0.0) { fprintf(stderr, "1x1 entropy %.17g, want 0\n", H); ++bad; }
  if (refused != MAXE_ERR_INVALID) { fprintf(stderr, "unknown flag: %s\n", maxe_status_str(refused)); ++bad; }

  CHECK_MAXE(maxe_handle_destroy(h));
  cudaFree(d_rowptr); cudaFree(d_col); cudaFree(d_val); cudaFree(d_rperm); cudaFree(d_cperm);
  cudaFree(d_x); cudaFree(d_y); cudaFree(d_x2);
  free(rowptr); free(col); free(val); free(x); free(y); free(y2);
  printf("maxe %s: n=%d seed=%llu, %d wrong\n", maxe_version(), n, (unsigned long long)seed, bad);
  return bad ? 1 : 0;
}
