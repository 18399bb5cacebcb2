// internal.cuh -- shared plumbing of libmaxe.so (not part of the ABI).
//
// Device side: inline-PTX wrappers for mbarriers, bulk (TMA) copies and
// bounded waits.  Host side: error macros, the scratch allocator and the
// launcher declarations of every kernel family.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/maxe.h"

namespace maxe {

// ----------------------------------------------------------------- limits
constexpr int64_t kMaxIndex = 2147483647LL - 64;  // rows, cols, nnz bound
constexpr int kPadElems = 4096;  // col/val arrays owned by a handle are rounded up to this multiple
constexpr int kRowptrPad = 8;    // extra rowptr entries owned by a handle
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded device waits give up after 2 s (default)

// The per-device status word every waiting kernel gets (DeviceInfo::status).
constexpr unsigned kDevTimeout = 1u;
constexpr size_t kDevWordBytes = 16;

// ----------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; give up after lim ns
// (the launch's wait limit, a kernel parameter), record kDevTimeout in *status
// and return false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* status, uint64_t lim) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > lim) {
      atomicOr(status, kDevTimeout);
      return false;
    }
  }
}

// L2 eviction-priority policy for data streamed once.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// 1-D bulk copy global -> shared through the TMA unit, completion counted on
// `bar` (complete_tx).  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// Named barrier among `n` threads (id >= 1; id 0 is __syncthreads).
__device__ __forceinline__ void named_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier that also ANDs a predicate over the participating threads.
__device__ __forceinline__ bool named_bar_and(int id, int n, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return out != 0;
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

// ------------------------------------------------------------ host helpers
#define MAXE_CUDA_TRY(expr)                      \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return MAXE_ERR_CUDA; \
  } while (0)

#define MAXE_TRY(expr)                 \
  do {                                 \
    maxe_status _s = (expr);           \
    if (_s != MAXE_OK) return _s;      \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Runs a set-up step (kernel attributes, which belong to a device's context)
// once per device, under a lock: host threads may launch concurrently.
struct PerDeviceOnce {
  std::mutex mu;
  bool done[64] = {};
  template <typename F>
  maxe_status run(F&& f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MAXE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return MAXE_OK;
    const maxe_status s = f();
    if (s == MAXE_OK) done[dev] = true;
    return s;
  }
};

inline int64_t round_up(int64_t a, int64_t m) { return (a + m - 1) / m * m; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Per-device facts and the device status word (allocated once per device).
struct DeviceInfo {
  int device;
  int sms;
  unsigned* status;  // device word (kDevWordBytes): bits of kDev*, then the wait limit
};
maxe_status device_info(DeviceInfo* out);
// The wait limit (ns) of bounded device waits for kernels launched on `device`
// (maxe_set_wait_limit_ns; kWaitNs by default).
uint64_t wait_limit_ns(int device);
uint64_t wait_limit_ns();  // the current device's

// Scratch / owned allocations through a maxe_allocator (or cudaMallocAsync).
struct Allocator {
  maxe_allocator a{};
  bool custom = false;
  cudaStream_t stream = nullptr;
  Allocator() = default;
  Allocator(const maxe_allocator* al, cudaStream_t s) : stream(s) {
    if (al && al->alloc && al->free) {
      a = *al;
      custom = true;
    }
  }
  void* get(size_t bytes) const {
    if (bytes == 0) bytes = 256;
    if (custom) return a.alloc(bytes, a.ctx, stream);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p) const {
    if (!p) return;
    if (custom)
      a.free(p, a.ctx, stream);
    else
      cudaFreeAsync(p, stream);
  }
};

// Scope guard releasing scratch blocks on every exit path.
struct ScratchSet {
  const Allocator& al;
  void* ptrs[16];
  int n = 0;
  explicit ScratchSet(const Allocator& a) : al(a) {}
  template <typename T>
  T* get(size_t count) {
    if (n >= 16) return nullptr;
    void* p = al.get(count * sizeof(T));
    if (p) ptrs[n++] = p;
    return static_cast<T*>(p);
  }
  ~ScratchSet() {
    for (int i = n - 1; i >= 0; --i) al.put(ptrs[i]);
  }
};

// ------------------------------------------------------- kernel launchers
// scan.cu: exclusive prefix sum of int32 (values >= 0) with total, in place allowed.
size_t scan_scratch_elems(int64_t n);
maxe_status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_out,
                               int32_t* scratch, cudaStream_t st);
// *p = v on the stream.
maxe_status set_i32(int32_t* p, int32_t v, cudaStream_t st);
// gradient.cu: entries per row (axis 0) or per column (axis 1); the gradient-based
// permutation of n rows or columns from such a histogram.
maxe_status nnz_histogram_run(const int32_t* rowptr, const int32_t* col, int32_t M, int32_t N, int64_t Z, int axis,
                              int32_t* hist, cudaStream_t st);
maxe_status gradient_permutation_run(const int32_t* hist, int32_t n, uint64_t seed, int32_t tag, int32_t* perm,
                                     int32_t* pivot_out, const Allocator& al, cudaStream_t st);
// first[g] = min{ i in [0, npos) : pos[i] >= g*H + off } (npos if none), g in [0, nb].
maxe_status bucket_lower_bounds(const int32_t* pos, int64_t npos, int64_t H, int64_t off, int64_t nb,
                                int32_t* first, cudaStream_t st);

// perm.cu
size_t radix_scratch_bytes(int64_t n);
// Stable LSD sort of (key, val) pairs by the low `bits` key bits.  Result ends
// in keys/vals (the *_alt buffers are ping-pong space).
maxe_status radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt,
                             int64_t n, int bits, void* scratch, cudaStream_t st);
maxe_status launch_keys(uint64_t seed, int32_t n, int32_t tag, uint64_t* keys, int32_t* idx, cudaStream_t st);
maxe_status launch_invert(const int32_t* perm, int32_t n, int32_t* inv, cudaStream_t st);
maxe_status launch_gather(const int32_t* perm, int64_t n, int elem_bytes, int64_t row_elems, const void* in,
                          int64_t ld_in, void* out, int64_t ld_out, cudaStream_t st);
maxe_status launch_scatter(const int32_t* perm, int64_t n, int elem_bytes, const void* in, void* out,
                           cudaStream_t st);

}  // namespace maxe
