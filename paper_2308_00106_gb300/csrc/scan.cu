// scan.cu -- device-wide exclusive prefix sum (row pointers of the permuted
// CSR, Section 2; digit offsets of the radix sort) and the bucket lower-bound
// search that partitions sorted offsets into fixed-size buckets.
#include "internal.cuh"

namespace maxe {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096
constexpr int kPartialThreads = 1024;

__host__ __device__ constexpr int padded(int i) { return i + (i >> 5); }

// sums[b] = sum of tile b of `in`.
__global__ void __launch_bounds__(kScanThreads) scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                            int32_t* __restrict__ sums) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = base + threadIdx.x + i * kScanThreads;
    if (e < n) s += in[e];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  __shared__ int32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// In-place exclusive scan of sums[0..nb) by one CTA; total written to *total.
__global__ void __launch_bounds__(kPartialThreads) scan_partials(int32_t* sums, int64_t nb, int32_t* total) {
  __shared__ int32_t ws[kPartialThreads / 32];
  __shared__ int32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += kPartialThreads) {
    int64_t e = base + threadIdx.x;
    int32_t v = e < nb ? sums[e] : 0;
    int32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += u;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    int32_t wpre = 0;
    for (int k = 0; k < w; ++k) wpre += ws[k];
    int32_t carry = carry_s;
    if (e < nb) sums[e] = carry + wpre + inc - v;
    __syncthreads();
    if (threadIdx.x == kPartialThreads - 1) carry_s = carry + wpre + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry_s;
}

// out[e] = offsets[tile] + exclusive scan of in within the tile.
__global__ void __launch_bounds__(kScanThreads) scan_apply(const int32_t* in, int32_t* out, int64_t n,
                                                           const int32_t* __restrict__ offsets) {
  __shared__ int32_t tile[padded(kScanTile)];
  __shared__ int32_t ws[kScanThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int idx = threadIdx.x + i * kScanThreads;
    int64_t e = base + idx;
    tile[padded(idx)] = e < n ? in[e] : 0;
  }
  __syncthreads();
  int32_t v[kScanItems];
  int32_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = run;
    run += tile[padded(threadIdx.x * kScanItems + i)];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int32_t u = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int32_t pre = offsets[blockIdx.x] + inc - run;
  for (int k = 0; k < w; ++k) pre += ws[k];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) tile[padded(threadIdx.x * kScanItems + i)] = pre + v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int idx = threadIdx.x + i * kScanThreads;
    int64_t e = base + idx;
    if (e < n) out[e] = tile[padded(idx)];
  }
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__global__ void bucket_lb_kernel(const int32_t* __restrict__ pos, int64_t npos, int64_t H, int64_t off,
                                 int64_t nb, int32_t* __restrict__ first) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > npos) return;
  int64_t lo = (i == 0) ? 0 : floor_div(static_cast<int64_t>(pos[i - 1]) - off, H) + 1;
  int64_t hi = (i == npos) ? nb : floor_div(static_cast<int64_t>(pos[i]) - off, H);
  if (lo < 0) lo = 0;
  if (hi > nb) hi = nb;
  for (int64_t g = lo; g <= hi; ++g) first[g] = static_cast<int32_t>(i);
}

__global__ void set_i32_kernel(int32_t* p, int32_t v) { *p = v; }

}  // namespace

maxe_status set_i32(int32_t* p, int32_t v, cudaStream_t st) {
  set_i32_kernel<<<1, 1, 0, st>>>(p, v);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

size_t scan_scratch_elems(int64_t n) { return static_cast<size_t>(ceil_div(n > 0 ? n : 1, kScanTile)) + 1; }

maxe_status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_out, int32_t* scratch,
                               cudaStream_t st) {
  if (n <= 0) {
    if (total_out) MAXE_CUDA_TRY(cudaMemsetAsync(total_out, 0, sizeof(int32_t), st));
    return MAXE_OK;
  }
  const int64_t nb = ceil_div(n, kScanTile);
  int32_t* sums = scratch;
  int32_t* total = total_out ? total_out : scratch + nb;
  scan_reduce<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, n, sums);
  scan_partials<<<1, kPartialThreads, 0, st>>>(sums, nb, total);
  scan_apply<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, out, n, sums);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status bucket_lower_bounds(const int32_t* pos, int64_t npos, int64_t H, int64_t off, int64_t nb,
                                int32_t* first, cudaStream_t st) {
  const int64_t threads = npos + 1;
  bucket_lb_kernel<<<static_cast<unsigned>(ceil_div(threads, 256)), 256, 0, st>>>(pos, npos, H, off, nb, first);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace maxe
