// gradient.cu -- the gradient-based permutations (Section 5 and the appendix's
// list of randomisation formats): the nonzero histogram of the rows (or
// columns), the cut at its steepest step, a riffle of the two parts, and a
// random order inside each half of the shuffled deck.
//
//   histogram: rows from rowptr differences, columns by integer atomics (exact,
//              order-free).
//   pivot:     max over i of (|h[i+1] - h[i]|, -i) packed in 64 bits and
//              reduced with atomicMax, so the first steepest step wins whatever
//              the schedule; the cut is before element i+1.
//   order:     each half of the deck is sorted by the Section 3 keys of its
//              positions (the radix sort of perm.cu, once per half).
//   compose:   perm[new] = deck[order[new]], the riffle written in closed form:
//              with parts of a = pivot and b = n - pivot cards and m = min(a, b),
//              deck[d] = d/2 (d even) or pivot + d/2 (d odd) for d < 2m, then the
//              longer part's remainder in order.
#include <algorithm>

#include "internal.cuh"

namespace maxe {
namespace {

constexpr int kThreads = 256;

__global__ void row_hist_kernel(const int32_t* __restrict__ rowptr, int32_t M, int32_t* __restrict__ hist) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < M) hist[i] = rowptr[i + 1] - rowptr[i];
}

__global__ void col_hist_kernel(const int32_t* __restrict__ col, int64_t Z, int32_t* __restrict__ hist) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < Z;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(hist + col[e], 1);
}

__global__ void __launch_bounds__(kThreads) steepest_kernel(const int32_t* __restrict__ h, int32_t n,
                                                            unsigned long long* __restrict__ best) {
  unsigned long long b = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i + 1 < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t g = static_cast<int64_t>(h[i + 1]) - static_cast<int64_t>(h[i]);
    const unsigned long long steep = static_cast<unsigned long long>(g < 0 ? -g : g);
    const unsigned long long packed = (steep << 32) | (0xffffffffull - static_cast<unsigned long long>(i));
    b = packed > b ? packed : b;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, d);
    b = o > b ? o : b;
  }
  if ((threadIdx.x & 31) == 0 && b != 0) atomicMax(best, b);
}

__global__ void riffle_compose_kernel(const int32_t* __restrict__ order, int32_t n,
                                      const unsigned long long* __restrict__ best, int32_t* __restrict__ perm,
                                      int32_t* __restrict__ pivot_out) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int64_t pivot = n;
  if (n >= 2) pivot = static_cast<int64_t>(0xffffffffull - (*best & 0xffffffffull)) + 1;
  if (q == 0 && pivot_out) *pivot_out = static_cast<int32_t>(pivot);
  const int64_t a = pivot, b = n - pivot, m = a < b ? a : b;
  const int64_t d = order[q];
  int64_t old;
  if (d < 2 * m)
    old = (d & 1) ? pivot + (d >> 1) : (d >> 1);
  else
    old = a > b ? d - b : d;
  perm[q] = static_cast<int32_t>(old);
}

}  // namespace

maxe_status nnz_histogram_run(const int32_t* rowptr, const int32_t* col, int32_t M, int32_t N, int64_t Z, int axis,
                              int32_t* hist, cudaStream_t st) {
  if (axis == 0) {
    if (M == 0) return MAXE_OK;
    row_hist_kernel<<<static_cast<unsigned>(ceil_div(M, kThreads)), kThreads, 0, st>>>(rowptr, M, hist);
  } else {
    if (N == 0) return MAXE_OK;
    MAXE_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int32_t) * static_cast<size_t>(N), st));
    if (Z == 0) return MAXE_OK;
    const int64_t blocks = std::min<int64_t>(ceil_div(Z, kThreads), 152 * 16);
    col_hist_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(col, Z, hist);
  }
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status gradient_permutation_run(const int32_t* hist, int32_t n, uint64_t seed, int32_t tag, int32_t* perm,
                                     int32_t* pivot_out, const Allocator& al, cudaStream_t st) {
  if (n == 0) return pivot_out ? set_i32(pivot_out, 0, st) : MAXE_OK;
  const int32_t half = (n + 1) / 2;
  ScratchSet scratch(al);
  uint64_t* keys = scratch.get<uint64_t>(n);
  uint64_t* keys_alt = scratch.get<uint64_t>(half);
  int32_t* order = scratch.get<int32_t>(n);
  int32_t* vals_alt = scratch.get<int32_t>(half);
  void* rs = scratch.get<unsigned char>(radix_scratch_bytes(half));
  unsigned long long* best = scratch.get<unsigned long long>(1);
  if (!keys || !keys_alt || !order || !vals_alt || !rs || !best) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long), st));
  if (n >= 2) {
    const int64_t blocks = std::min<int64_t>(ceil_div(n, kThreads), 152 * 8);
    steepest_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, st>>>(hist, n, best);
    MAXE_CUDA_TRY(cudaGetLastError());
  }
  MAXE_TRY(launch_keys(seed, n, tag, keys, order, st));  // keys of the deck positions, order = positions
  MAXE_TRY(radix_sort_pairs(keys, order, keys_alt, vals_alt, half, 64, rs, st));
  MAXE_TRY(radix_sort_pairs(keys + half, order + half, keys_alt, vals_alt, n - half, 64, rs, st));
  riffle_compose_kernel<<<static_cast<unsigned>(ceil_div(n, kThreads)), kThreads, 0, st>>>(order, n, best, perm,
                                                                                         pivot_out);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace maxe
