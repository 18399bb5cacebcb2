// entropy.cu -- entropy of the nonzero distribution (Section 4, entropy
// equation) over a gr x gc block grid of the matrix (Section 5's 2-D
// histograms / hierarchical grids).
//
// bin(i, j) = (floor(i*gr/M), floor(j*gc/N)) with 64-bit products.
// Row bin b covers rows [ceil(b*M/gr), ceil((b+1)*M/gr)), i.e. the contiguous
// entry range [E_b, E_{b+1}) with E_b = rowptr[ceil(b*M/gr)].  So the
// histogram is entry-parallel: each CTA takes 8192 consecutive entries, finds
// the few row bins they span (binary search over E), counts (row bin, column
// bin) pairs in shared memory (or global memory for wide grids) and adds its
// counts to a global table.  One CTA then forms H = -sum_{c>0} p log_base p in
// FP64 in a fixed order (deterministic).  Only rowptr and col are read:
// 4 bytes per entry plus the row pointers.
#include <algorithm>
#include <mutex>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kHThreads = 256;
constexpr int kHItems = 32;
constexpr int kHTile = kHThreads * kHItems;  // 8192 entries per CTA
constexpr int kHMaxBins = 8192;              // shared-memory bins per CTA
constexpr int kHMaxRowBins = 512;            // row-bin edges held in shared memory

__device__ __forceinline__ int64_t row_bin_start(int64_t b, int64_t M, int64_t gr) {
  return (b * M + gr - 1) / gr;  // ceil(b*M/gr)
}

// E_b = first entry of row bin b
__device__ __forceinline__ int64_t edge(const int32_t* rowptr, int64_t b, int64_t M, int64_t gr) {
  return rowptr[row_bin_start(b, M, gr)];
}

// largest b in [lo, hi] with E_b <= e (E_lo <= e assumed)
__device__ __forceinline__ int64_t find_bin(const int32_t* rowptr, int64_t e, int64_t lo, int64_t hi, int64_t M,
                                            int64_t gr) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (edge(rowptr, mid, M, gr) <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kHThreads) hist_kernel(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col, int32_t M, int32_t N,
                                                         int64_t Z, int32_t gr, int32_t gc,
                                                         unsigned* __restrict__ counts) {
  __shared__ unsigned hist[kHMaxBins];
  __shared__ int32_t edges[kHMaxRowBins + 1];
  __shared__ int64_t blo_s, bhi_s;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kHTile;
  const int64_t last = std::min<int64_t>(base + kHTile, Z) - 1;
  if (threadIdx.x == 0) {
    blo_s = find_bin(rowptr, base, 0, gr - 1, M, gr);
    bhi_s = find_bin(rowptr, last, blo_s, gr - 1, M, gr);
  }
  __syncthreads();
  const int64_t blo = blo_s, bhi = bhi_s;
  const int64_t nrb = bhi - blo + 1;
  const bool edges_in_smem = nrb <= kHMaxRowBins;
  const bool bins_in_smem = nrb * gc <= kHMaxBins;
  if (edges_in_smem)
    for (int64_t t = threadIdx.x; t <= nrb; t += kHThreads)
      edges[t] = (blo + t <= gr) ? static_cast<int32_t>(edge(rowptr, blo + t, M, gr)) : static_cast<int32_t>(Z);
  if (bins_in_smem)
    for (int64_t t = threadIdx.x; t < nrb * gc; t += kHThreads) hist[t] = 0u;
  __syncthreads();
  int64_t cur = 0;  // row bin of the previous entry, relative to blo (entries of a thread increase)
  for (int i = 0; i < kHItems; ++i) {
    const int64_t e = base + threadIdx.x + static_cast<int64_t>(i) * kHThreads;
    if (e > last) break;
    int64_t rb;
    if (edges_in_smem) {
      while (cur + 1 < nrb && edges[cur + 1] <= e) ++cur;
      rb = cur;
    } else {
      rb = find_bin(rowptr, e, blo, bhi, M, gr) - blo;
    }
    const int64_t cb = static_cast<int64_t>(col[e]) * gc / N;
    if (bins_in_smem)
      atomicAdd(&hist[rb * gc + cb], 1u);
    else
      atomicAdd(&counts[(blo + rb) * gc + cb], 1u);
  }
  if (bins_in_smem) {
    __syncthreads();
    for (int64_t t = threadIdx.x; t < nrb * gc; t += kHThreads) {
      const unsigned c = hist[t];
      if (c) atomicAdd(&counts[blo * gc + t], c);
    }
  }
}

constexpr int kEThreads = 1024;

__global__ void __launch_bounds__(kEThreads) entropy_kernel(const unsigned* __restrict__ counts, int64_t nbins,
                                                            int64_t Z, double base, int64_t* __restrict__ counts64,
                                                            double* __restrict__ H) {
  __shared__ double ws[kEThreads / 32];
  const double inv_lb = (base == 2.0) ? 1.0 : 1.0 / log(base);
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < nbins; b += kEThreads) {
    const unsigned c = counts[b];
    if (counts64) counts64[b] = static_cast<int64_t>(c);
    if (c && Z > 0) {
      const double pr = static_cast<double>(c) / static_cast<double>(Z);
      acc -= pr * ((base == 2.0) ? log2(pr) : log(pr) * inv_lb);
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEThreads / 32; ++w) t += ws[w];
    *H = t;
  }
}

// Hierarchical 2-D entropy: one CTA per cell (a, b) of an L x L split of the
// count grid; the cell's total, then -sum p log p, both reduced in a fixed order.
constexpr int kLThreads = 256;

__global__ void __launch_bounds__(kLThreads) entropy_levels_kernel(const int64_t* __restrict__ counts, int32_t gr,
                                                                   int32_t gc, int32_t L, double base,
                                                                   double* __restrict__ out) {
  __shared__ double ws[kLThreads / 32];
  __shared__ long long wt[kLThreads / 32];
  const int a = blockIdx.x / L, b = blockIdx.x - (blockIdx.x / L) * L;
  const int64_t r0 = (static_cast<int64_t>(a) * gr + L - 1) / L, r1 = (static_cast<int64_t>(a + 1) * gr + L - 1) / L;
  const int64_t c0 = (static_cast<int64_t>(b) * gc + L - 1) / L, c1 = (static_cast<int64_t>(b + 1) * gc + L - 1) / L;
  const int64_t w = c1 - c0, n = (r1 - r0) * w;
  long long t = 0;
  for (int64_t i = threadIdx.x; i < n; i += kLThreads) t += counts[(r0 + i / w) * gc + c0 + i % w];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
  if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = t;
  __syncthreads();
  long long S = 0;
  for (int k = 0; k < kLThreads / 32; ++k) S += wt[k];
  double acc = 0.0;
  if (S > 0) {
    const double inv_lb = (base == 2.0) ? 1.0 : 1.0 / log(base);
    for (int64_t i = threadIdx.x; i < n; i += kLThreads) {
      const long long c = counts[(r0 + i / w) * gc + c0 + i % w];
      if (c == 0) continue;
      const double pr = static_cast<double>(c) / static_cast<double>(S);
      acc -= pr * ((base == 2.0) ? log2(pr) : log(pr) * inv_lb);
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double H = 0.0;
    for (int k = 0; k < kLThreads / 32; ++k) H += ws[k];
    out[blockIdx.x] = H;
  }
}

}  // namespace

maxe_status entropy_run(const maxe_handle* h, int32_t gr, int32_t gc, double base, double* H_host,
                        int64_t* counts_dev, const Allocator& al, cudaStream_t st) {
  const int64_t nbins = static_cast<int64_t>(gr) * gc;
  ScratchSet scratch(al);
  unsigned* counts = scratch.get<unsigned>(static_cast<size_t>(nbins));
  double* Hd = scratch.get<double>(1);
  if (!counts || !Hd) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(unsigned) * nbins, st));
  if (h->nnz > 0) {
    const int64_t grid = ceil_div(h->nnz, kHTile);
    hist_kernel<<<static_cast<unsigned>(grid), kHThreads, 0, st>>>(h->rowptr, h->col, h->rows, h->cols, h->nnz, gr,
                                                                    gc, counts);
    MAXE_CUDA_TRY(cudaGetLastError());
  }
  entropy_kernel<<<1, kEThreads, 0, st>>>(counts, nbins, h->nnz, base, counts_dev, Hd);
  MAXE_CUDA_TRY(cudaGetLastError());
  MAXE_CUDA_TRY(cudaMemcpyAsync(H_host, Hd, sizeof(double), cudaMemcpyDeviceToHost, st));
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  return MAXE_OK;
}

}  // namespace maxe

extern "C" maxe_status maxe_entropy_levels(const int64_t* counts_dev, int32_t gr, int32_t gc, int32_t L, double base,
                                           double* H_dev, void* stream) {
  using namespace maxe;
  if (!counts_dev || !H_dev || gr < 1 || gc < 1 || L < 1 || L > gr || L > gc || !(base > 1.0) || L > 4096)
    return MAXE_ERR_INVALID;
  entropy_levels_kernel<<<static_cast<unsigned>(L) * L, kLThreads, 0, as_stream(stream)>>>(counts_dev, gr, gc, L,
                                                                                             base, H_dev);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

// ------------------------------------------------- allocation-free variant
namespace {

constexpr int64_t kNoAllocMaxBins = 65536;  // grid cells the static scratch holds (256 KiB of counts)

// Scratch of maxe_nnz_entropy_noalloc: kNoAllocMaxBins 32-bit counts, then H.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_entropy_scratch[kNoAllocMaxBins * sizeof(unsigned) + 256];

// The current context's id (driver calls resolved through the runtime, no
// link to the driver library); 0 when it cannot be had.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_entropy_scratch, looked up on a device's first call with
// that device current (in host code the symbol is only a host-side stand-in).
// The address belongs to the device's context: a call after the context was
// torn down and made again (cudaDeviceReset) looks it up again.
maxe_status noalloc_scratch(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[64] = {};
  static unsigned long long ctx_of[64] = {};
  int dev = 0;
  MAXE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MAXE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long ctx = current_context_id();
  if (!addr[dev] || (ctx != 0 && ctx != ctx_of[dev])) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_entropy_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MAXE_ERR_CUDA;
    }
    addr[dev] = static_cast<unsigned char*>(p);
    ctx_of[dev] = ctx != 0 ? ctx : current_context_id();  // the lookup made the context current if it was not
  }
  *out = addr[dev];
  return MAXE_OK;
}

}  // namespace

extern "C" maxe_status maxe_nnz_entropy_noalloc(const maxe_handle* h, int32_t gr, int32_t gc, double base,
                                                double* H_host, int64_t* counts_dev, void* stream) {
  using namespace maxe;
  if (!h || !H_host) return MAXE_ERR_INVALID;
  if (gr < 1 || gc < 1 || gr > h->rows || gc > h->cols || !(base > 1.0)) return MAXE_ERR_INVALID;
  const int64_t nbins = static_cast<int64_t>(gr) * gc;
  if (nbins > kNoAllocMaxBins) return MAXE_ERR_INVALID;
  unsigned char* scratch = nullptr;
  MAXE_TRY(noalloc_scratch(&scratch));
  unsigned* counts = reinterpret_cast<unsigned*>(scratch);
  double* Hd = reinterpret_cast<double*>(scratch + kNoAllocMaxBins * sizeof(unsigned));
  cudaStream_t st = as_stream(stream);
  // the array keeps the previous call's counts: clear the cells this call uses
  MAXE_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(unsigned) * nbins, st));
  if (h->nnz > 0) {
    const int64_t grid = ceil_div(h->nnz, kHTile);
    hist_kernel<<<static_cast<unsigned>(grid), kHThreads, 0, st>>>(h->rowptr, h->col, h->rows, h->cols, h->nnz, gr,
                                                                    gc, counts);
    MAXE_CUDA_TRY(cudaGetLastError());
  }
  entropy_kernel<<<1, kEThreads, 0, st>>>(counts, nbins, h->nnz, base, counts_dev, Hd);
  MAXE_CUDA_TRY(cudaGetLastError());
  MAXE_CUDA_TRY(cudaMemcpyAsync(H_host, Hd, sizeof(double), cudaMemcpyDeviceToHost, st));
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  return MAXE_OK;
}
