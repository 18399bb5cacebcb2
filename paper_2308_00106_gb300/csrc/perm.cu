// perm.cu -- the random permutation of Section 3 and the vector permutations
// of Eq. 1.
//
//   keys:   key(seed, tag, i) = output number 2i+tag+1 of SplitMix64 seeded with
//           `seed` (Steele, Lea, Flood 2014), one thread per index.
//   sort:   stable LSD radix sort of (key, index) pairs, 8 bits per pass; the
//           sorted indices are perm[new] = old.  Stability breaks key ties by index.
//   invert: inv[perm[i]] = i.
//   gather / scatter: x' = P_c^{-1} x and y = P_r^{-1} y'.
#include "internal.cuh"

namespace maxe {
namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ull;

__device__ __forceinline__ uint64_t splitmix_output(uint64_t seed, uint64_t m) {
  uint64_t z = seed + m * kGamma;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void keys_kernel(uint64_t seed, int32_t n, int32_t tag, uint64_t* __restrict__ keys,
                            int32_t* __restrict__ idx) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = splitmix_output(seed, 2ull * static_cast<uint64_t>(i) + static_cast<uint64_t>(tag) + 1ull);
  idx[i] = static_cast<int32_t>(i);
}

// ------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096 keys per tile
constexpr int kRsWarpKeys = 32 * kRsItems;      // 512 keys per warp
constexpr int kBins = 256;

// counts[d * ntiles + tile] = number of keys of the tile with digit d.
__global__ void __launch_bounds__(kRsThreads) rs_upsweep(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                         int32_t* __restrict__ counts, int64_t ntiles) {
  __shared__ uint32_t hist[kBins];
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kRsTile;
#pragma unroll 4
  for (int i = 0; i < kRsItems; ++i) {
    int64_t e = base + threadIdx.x + i * kRsThreads;
    if (e < n) atomicAdd(&hist[(keys[e] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  counts[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x] = static_cast<int32_t>(hist[threadIdx.x]);
}

// Stable scatter of one tile: warp w owns keys [w*512, w*512+512) of the tile,
// visited 32 at a time in index order, so rank order equals index order.
__global__ void __launch_bounds__(kRsThreads) rs_scatter(const uint64_t* __restrict__ kin,
                                                         const int32_t* __restrict__ vin,
                                                         uint64_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                         int64_t n, int shift, const int32_t* __restrict__ offs,
                                                         int64_t ntiles) {
  __shared__ uint32_t wcount[kRsWarps][kBins];
  __shared__ uint32_t tile_off[kBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * kBins; i += kRsThreads) (&wcount[0][0])[i] = 0;
  tile_off[threadIdx.x] = static_cast<uint32_t>(offs[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x]);
  __syncthreads();

  const int64_t base = static_cast<int64_t>(blockIdx.x) * kRsTile + w * kRsWarpKeys;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t k[kRsItems];
  int32_t v[kRsItems];
  uint32_t rank[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t e = base + j * 32 + lane;
    const bool valid = e < n;
    k[j] = valid ? kin[e] : 0ull;
    v[j] = valid ? vin[e] : 0;
    const uint32_t d = valid ? static_cast<uint32_t>((k[j] >> shift) & 0xFF) : static_cast<uint32_t>(kBins);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (valid && lane == leader) {
      old = wcount[w][d];
      wcount[w][d] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[j] = old + __popc(peers & lt_mask);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix over warps, per digit
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ++ww) {
      uint32_t t = wcount[ww][d];
      wcount[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t e = base + j * 32 + lane;
    if (e < n) {
      const uint32_t d = static_cast<uint32_t>((k[j] >> shift) & 0xFF);
      const int64_t pos = static_cast<int64_t>(tile_off[d]) + wcount[w][d] + rank[j];
      kout[pos] = k[j];
      vout[pos] = v[j];
    }
  }
}

__global__ void invert_kernel(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ inv) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) inv[perm[i]] = static_cast<int32_t>(i);
}

template <typename T>
__global__ void gather_kernel(const int32_t* __restrict__ perm, int64_t n, int64_t row_elems,
                              const T* __restrict__ in, int64_t ld_in, T* __restrict__ out, int64_t ld_out) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * row_elems) return;
  const int64_t i = t / row_elems, c = t - i * row_elems;
  out[i * ld_out + c] = in[static_cast<int64_t>(perm[i]) * ld_in + c];
}

template <typename T>
__global__ void scatter_kernel(const int32_t* __restrict__ perm, int64_t n, const T* __restrict__ in,
                               T* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[perm[i]] = in[i];
}

}  // namespace

size_t radix_scratch_bytes(int64_t n) {
  const int64_t ntiles = ceil_div(n > 0 ? n : 1, kRsTile);
  const int64_t counts = kBins * ntiles;
  return static_cast<size_t>(counts + static_cast<int64_t>(scan_scratch_elems(counts))) * sizeof(int32_t);
}

maxe_status radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, int64_t n,
                             int bits, void* scratch, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return MAXE_OK;
  const int64_t ntiles = ceil_div(n, kRsTile);
  int32_t* counts = static_cast<int32_t*>(scratch);
  int32_t* scan_tmp = counts + kBins * ntiles;
  const int passes = (bits + 7) / 8;
  uint64_t* kin = keys;
  int32_t* vin = vals;
  uint64_t* kout = keys_alt;
  int32_t* vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    rs_upsweep<<<static_cast<unsigned>(ntiles), kRsThreads, 0, st>>>(kin, n, shift, counts, ntiles);
    MAXE_TRY(scan_exclusive_i32(counts, counts, kBins * ntiles, nullptr, scan_tmp, st));
    rs_scatter<<<static_cast<unsigned>(ntiles), kRsThreads, 0, st>>>(kin, vin, kout, vout, n, shift, counts,
                                                                      ntiles);
    MAXE_CUDA_TRY(cudaGetLastError());
    uint64_t* tk = kin;
    kin = kout;
    kout = tk;
    int32_t* tv = vin;
    vin = vout;
    vout = tv;
  }
  if (kin != keys) {  // odd number of passes: bring the result home
    MAXE_CUDA_TRY(cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    MAXE_CUDA_TRY(cudaMemcpyAsync(vals, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  }
  return MAXE_OK;
}

maxe_status launch_keys(uint64_t seed, int32_t n, int32_t tag, uint64_t* keys, int32_t* idx, cudaStream_t st) {
  if (n <= 0) return MAXE_OK;
  keys_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(seed, n, tag, keys, idx);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status launch_invert(const int32_t* perm, int32_t n, int32_t* inv, cudaStream_t st) {
  if (n <= 0) return MAXE_OK;
  invert_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(perm, n, inv);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status launch_gather(const int32_t* perm, int64_t n, int elem_bytes, int64_t row_elems, const void* in,
                          int64_t ld_in, void* out, int64_t ld_out, cudaStream_t st) {
  const int64_t total = n * row_elems;
  if (total <= 0) return MAXE_OK;
  const unsigned grid = static_cast<unsigned>(ceil_div(total, 256));
  switch (elem_bytes) {
    case 2:
      gather_kernel<uint16_t><<<grid, 256, 0, st>>>(perm, n, row_elems, static_cast<const uint16_t*>(in), ld_in,
                                                   static_cast<uint16_t*>(out), ld_out);
      break;
    case 4:
      gather_kernel<uint32_t><<<grid, 256, 0, st>>>(perm, n, row_elems, static_cast<const uint32_t*>(in), ld_in,
                                                   static_cast<uint32_t*>(out), ld_out);
      break;
    case 8:
      gather_kernel<uint64_t><<<grid, 256, 0, st>>>(perm, n, row_elems, static_cast<const uint64_t*>(in), ld_in,
                                                   static_cast<uint64_t*>(out), ld_out);
      break;
    default:
      return MAXE_ERR_INVALID;
  }
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status launch_scatter(const int32_t* perm, int64_t n, int elem_bytes, const void* in, void* out,
                           cudaStream_t st) {
  if (n <= 0) return MAXE_OK;
  const unsigned grid = static_cast<unsigned>(ceil_div(n, 256));
  switch (elem_bytes) {
    case 2:
      scatter_kernel<uint16_t><<<grid, 256, 0, st>>>(perm, n, static_cast<const uint16_t*>(in),
                                                    static_cast<uint16_t*>(out));
      break;
    case 4:
      scatter_kernel<uint32_t><<<grid, 256, 0, st>>>(perm, n, static_cast<const uint32_t*>(in),
                                                    static_cast<uint32_t*>(out));
      break;
    case 8:
      scatter_kernel<uint64_t><<<grid, 256, 0, st>>>(perm, n, static_cast<const uint64_t*>(in),
                                                    static_cast<uint64_t*>(out));
      break;
    default:
      return MAXE_ERR_INVALID;
  }
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace maxe
