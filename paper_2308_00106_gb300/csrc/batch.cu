// batch.cu -- batched persistent SpMV/SpMM: many permuted matrices, each with
// its own k right-hand sides, in one persistent launch per value type and
// kernel class present.
//
// Each item is (handle, k, X, ldx, Y, ldy): Y = A' X with X in the permuted
// space, Y written in the permuted space or, with MAXE_BATCH_SCATTER_Y,
// through rperm into the original space.  Every handle carries a batch plan
// (entries per warp task H_b and entries per lane), built once per handle
// (default or tuned by maxe_batch_tune) and independent of what else is in a
// batch, so a matrix gives the same bits alone and in any mix.
//
// The launch keeps (blocks per SM x SMs) blocks resident; every warp takes
// tasks (item, warp range) from a flat list (first by position, then from an
// atomic counter, so uneven tasks balance out), runs each range
// through the same per-warp TMA ring as the single-matrix kernel (the ring's
// mbarrier phase count carries over between tasks), and picks the kernel
// variant (VW columns per pass, 8 or 16 entries per lane) per item.  A batch
// object stages its descriptor table in pinned host memory and uploads it on
// the stream before the launch, so batch runs can be captured in a CUDA graph.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "spmm_rows.cuh"
#include "spmv_warp.cuh"

namespace maxe {
namespace {

using namespace warp;

struct BatchItem {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  const void* X;
  void* Y;
  const int32_t* yperm;
  const int32_t* wrow;
  int64_t ldx, ldy;
  int32_t k, M, nW, vw, it16, unit, lcg;
};

struct BatchParams {
  const BatchItem* items;
  const int32_t* task0;  // first task of each item, nitems + 1 entries
  unsigned* status;
  int32_t* next;         // dynamic task counter (zeroed before the launch)
  int32_t nitems, ntasks;
  uint64_t wait_ns;      // limit of the bounded waits
};

// Kernel classes: register budgets differ a lot between the variants, so each
// class is its own persistent kernel (one launch per value type and class
// present in a batch): 0 = plain SpMV (k = 1, unit strides), 8 entries per
// lane; 1 = the same with 16 entries per lane; 2 = SpMM (1, 2 or 4 columns per
// pass, or columns across lanes, any strides); 3 = SpMM with one row per lane
// group (spmm_rows.cuh: 16-byte aligned X and Y rows).
constexpr int kClasses = 4;

template <typename VT, int CLASS>
struct BatchClass {
  static constexpr int kMinBlocks = CLASS == 0 ? 3 : 2;  // class 0 at 4 blocks spills (64 registers)
  static constexpr size_t warp_smem() {
    size_t m = 0;
    if (CLASS == 0) m = sizeof(WarpSmem<VT, 1, 8>);
    if (CLASS == 1) m = sizeof(WarpSmem<VT, 1, 16>);
    if (CLASS == 2) {
      m = std::max(sizeof(WarpSmem<VT, 1, 8>), sizeof(WarpSmem<VT, 2, 8>));
      m = std::max(m, sizeof(WarpSmemLC<VT>));
      if (sizeof(typename Acc<VT>::T) == 4) m = std::max(m, sizeof(WarpSmem<VT, 4, 8>));
    }
    if (CLASS == 3) m = sizeof(rows::RowsStage<VT>);
    return (m + 127) & ~size_t(127);
  }
};

template <typename VT, int CLASS>
__global__ void __launch_bounds__(kThreads, BatchClass<VT, CLASS>::kMinBlocks) spmm_batch_kernel(BatchParams bp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  unsigned char* wsmem = smem_raw + BatchClass<VT, CLASS>::warp_smem() * wib;
  init_ring<Cfg<VT, 1, 8, true>>(wsmem);  // barriers sit at offset 0 in every variant
  uint32_t gi = 0;
  const int nwarps = gridDim.x * kWarps;
  // first task by position, then the next unclaimed one (tasks differ in cost)
  for (int t = blockIdx.x * kWarps + wib; t < bp.ntasks;) {
    int lo = 0, hi = bp.nitems - 1;  // item of task t: last item with task0 <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bp.task0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const BatchItem& it = bp.items[lo];
    Params p;
    p.rowptr = it.rowptr;
    p.col = it.col;
    p.val = it.val;
    p.X = it.X;
    p.Y = it.Y;
    p.yperm = it.yperm;
    p.wrow = it.wrow;
    p.status = bp.status;
    p.wait_ns = bp.wait_ns;
    p.ldx = it.ldx;
    p.ldy = it.ldy;
    p.k = it.k;
    p.M = it.M;
    p.nW = it.nW;
    const int w = t - bp.task0[lo];
    bool ok = false;
    if constexpr (CLASS == 0) {
      ok = process_range<Cfg<VT, 1, 8, true>>(p, w, wsmem, gi);
    } else if constexpr (CLASS == 1) {
      ok = process_range<Cfg<VT, 1, 16, true>>(p, w, wsmem, gi);
    } else {
      if (it.lcg > 0) {
        ok = process_range_lc<VT>(p, w, wsmem, gi, it.lcg);
      } else if (it.vw == 1) {
        ok = process_range<Cfg<VT, 1, 8, false>>(p, w, wsmem, gi);
      } else if (it.vw == 2) {
        ok = process_range<Cfg<VT, 2, 8, false>>(p, w, wsmem, gi);
      } else {
        if constexpr (sizeof(typename Acc<VT>::T) == 4) ok = process_range<Cfg<VT, 4, 8, false>>(p, w, wsmem, gi);
      }
    }
    if (!ok) return;
    int nt = 0;
    if ((threadIdx.x & 31) == 0) nt = nwarps + atomicAdd(bp.next, 1);
    t = __shfl_sync(0xffffffffu, nt, 0);
  }
}

// Class 3: each warp task (item, warp range of the item's batch plan) runs
// the rows of its range through the chunk pipeline of spmm_rows.cuh, G lanes
// per row as the item's k asks.
template <typename VT>
__global__ void __launch_bounds__(kThreads) spmm_batch_rows_kernel(BatchParams bp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  rows::RowsStage<VT>* s =
      reinterpret_cast<rows::RowsStage<VT>*>(smem_raw + BatchClass<VT, 3>::warp_smem() * wib);
  const int nwarps = gridDim.x * kWarps;
  for (int t = blockIdx.x * kWarps + wib; t < bp.ntasks;) {
    int lo = 0, hi = bp.nitems - 1;  // item of task t: last item with task0 <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bp.task0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const BatchItem& it = bp.items[lo];
    const rows::RowsOperand op{it.rowptr, it.col, it.val, it.X, it.Y, it.yperm, it.ldx, it.ldy, it.k, 0};
    const int w = t - bp.task0[lo];
    rows::rows_range<VT>(s, op, it.wrow[w], it.wrow[w + 1], rows::rows_group<VT>(it.k), lane);
    int nt = 0;
    if (lane == 0) nt = nwarps + atomicAdd(bp.next, 1);
    t = __shfl_sync(0xffffffffu, nt, 0);
  }
}

template <typename VT, int CLASS>
constexpr auto batch_kernel() {
  if constexpr (CLASS == 3)
    return spmm_batch_rows_kernel<VT>;
  else
    return spmm_batch_kernel<VT, CLASS>;
}

// class of an item (see above); rows: the item takes the rows kernel
int item_class(int vw, int unit, int it16, bool rows) { return unit ? (it16 ? 1 : 0) : (rows ? 3 : 2); }

template <typename VT, int CLASS>
maxe_status batch_prepare(int* blocks_per_sm) {
  static PerDeviceOnce once;  // the attribute and the occupancy are per device
  static int occ[64] = {};
  int dev = 0;
  MAXE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MAXE_ERR_UNSUPPORTED;
  MAXE_TRY(once.run([dev] {
    const size_t smem = BatchClass<VT, CLASS>::warp_smem() * kWarps;
    MAXE_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<VT, CLASS>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
    int o = 0;
    MAXE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, batch_kernel<VT, CLASS>(), kThreads, smem));
    occ[dev] = o > 0 ? o : 1;
    return MAXE_OK;
  }));
  *blocks_per_sm = occ[dev];
  return MAXE_OK;
}

// bps: CTAs per SM (0: as many as fit).  The grid only changes which warp
// takes which task, never a task's sums: results do not depend on it.
template <typename VT, int CLASS>
maxe_status batch_launch(const BatchParams& bp, int sms, int bps, cudaStream_t st) {
  int occ = 1;
  MAXE_TRY((batch_prepare<VT, CLASS>(&occ)));
  if (bps > 0 && bps < occ) occ = bps;
  const int64_t want = ceil_div(bp.ntasks, kWarps);
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * occ)));
  batch_kernel<VT, CLASS>()<<<grid, kThreads, BatchClass<VT, CLASS>::warp_smem() * kWarps, st>>>(bp);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status batch_launch_class(int cls, const BatchParams& bp, int sms, int bps, cudaStream_t st) {
  if (cls == 0) return batch_launch<VT, 0>(bp, sms, bps, st);
  if (cls == 1) return batch_launch<VT, 1>(bp, sms, bps, st);
  if (cls == 2) return batch_launch<VT, 2>(bp, sms, bps, st);
  return batch_launch<VT, 3>(bp, sms, bps, st);
}

maxe_status launch_for(maxe_dtype d, int cls, const BatchParams& bp, int sms, int bps, cudaStream_t st) {
  switch (d) {
    case MAXE_F64: return batch_launch_class<double>(cls, bp, sms, bps, st);
    case MAXE_F32: return batch_launch_class<float>(cls, bp, sms, bps, st);
    case MAXE_BF16: return batch_launch_class<uint16_t>(cls, bp, sms, bps, st);
  }
  return MAXE_ERR_INVALID;
}

// CTAs per SM that the batched kernel of (value type, class) fits
int batch_occupancy(maxe_dtype d, int cls) {
  int occ = 1;
  maxe_status s = MAXE_OK;
  auto one = [&](auto vt) {
    using VT = decltype(vt);
    if (cls == 0) s = batch_prepare<VT, 0>(&occ);
    else if (cls == 1) s = batch_prepare<VT, 1>(&occ);
    else if (cls == 2) s = batch_prepare<VT, 2>(&occ);
    else s = batch_prepare<VT, 3>(&occ);
  };
  switch (d) {
    case MAXE_F64: one(double{}); break;
    case MAXE_F32: one(float{}); break;
    case MAXE_BF16: one(uint16_t{}); break;
  }
  return s == MAXE_OK ? occ : 1;
}

// resident warps of the batched kernel (class 0) for one value type
int batch_resident_warps(maxe_dtype d, int sms) {
  int occ = 1;
  maxe_status s = MAXE_OK;
  switch (d) {
    case MAXE_F64: s = batch_prepare<double, 0>(&occ); break;
    case MAXE_F32: s = batch_prepare<float, 0>(&occ); break;
    case MAXE_BF16: s = batch_prepare<uint16_t, 0>(&occ); break;
  }
  if (s != MAXE_OK) occ = 1;
  return sms * occ * kWarps;
}

int pick_vw(const maxe_batch_item& a, int eb) {
  if (a.k == 1) return 1;
  auto aligned = [&](int vw) {
    const uintptr_t al = static_cast<uintptr_t>(vw) * eb;
    return a.ldx % vw == 0 && a.ldy % vw == 0 && reinterpret_cast<uintptr_t>(a.X) % al == 0 &&
           reinterpret_cast<uintptr_t>(a.Y) % al == 0;
  };
  if (eb == 4 && a.k >= 3 && aligned(4)) return 4;
  if (aligned(2)) return 2;
  return 1;
}

}  // namespace

// Batch plan of a handle: a partition with H_b entries per warp task.
maxe_status batch_plan(maxe_handle* h, int64_t H, int it16, cudaStream_t st, int lc, int bps) {
  H = std::max<int64_t>(256, H);
  const int64_t nW = std::max<int64_t>(1, ceil_div(h->nnz, H));
  int32_t* w = static_cast<int32_t*>(h->al.get(static_cast<size_t>(nW + 1) * sizeof(int32_t)));
  if (!w) return MAXE_ERR_OOM;
  maxe_status s = bucket_lower_bounds(h->rowptr, h->rows, H, 0, nW, w, st);
  if (s == MAXE_OK) s = set_i32(w + nW, h->rows, st);
  if (s != MAXE_OK) {
    h->al.put(w);
    return s;
  }
  h->al.put(h->bwrow);
  h->bwrow = w;
  h->bnW = static_cast<int32_t>(nW);
  h->bH = H;
  h->bit16 = it16;
  h->blc = lc;
  h->bbps = bps;
  return MAXE_OK;
}

maxe_status batch_plan_default(maxe_handle* h, cudaStream_t st) {
  const int64_t target = batch_resident_warps(h->dtype, h->sms);
  return batch_plan(h, std::max<int64_t>(kDefaultBatchTask, ceil_div(std::max<int64_t>(h->nnz, 1), target)), 0, st,
                    2);
}

}  // namespace maxe

using namespace maxe;

struct maxe_batch {
  int32_t capacity = 0;
  int32_t n = 0;
  Allocator al;
  int sms = 0;
  unsigned* status = nullptr;
  // per value type: host staging (pinned) and device tables
  BatchItem* h_items = nullptr;
  int32_t* h_task0 = nullptr;
  BatchItem* d_items = nullptr;
  int32_t* d_task0 = nullptr;
  int32_t* d_next = nullptr;  // one dynamic task counter per (value type, class) group
  cudaEvent_t uploaded = nullptr;  // the last upload from the staging has executed
  bool pending = false;
  std::vector<maxe_batch_item> items;
};

namespace {

void batch_release(maxe_batch* b) {
  if (!b) return;
  if (b->uploaded) {
    cudaEventSynchronize(b->uploaded);
    cudaEventDestroy(b->uploaded);
  }
  b->al.put(b->d_next);
  b->al.put(b->d_task0);
  b->al.put(b->d_items);
  if (b->h_task0) cudaFreeHost(b->h_task0);
  if (b->h_items) cudaFreeHost(b->h_items);
  delete b;
}

}  // namespace

extern "C" {

maxe_status maxe_batch_create(int32_t capacity, const maxe_allocator* alloc, void* stream, maxe_batch** out) {
  if (!out || capacity < 1 || capacity > (1 << 20)) return MAXE_ERR_INVALID;
  *out = nullptr;
  DeviceInfo di{};
  MAXE_TRY(device_info(&di));
  cudaStream_t st = as_stream(stream);
  maxe_batch* b = new (std::nothrow) maxe_batch();
  if (!b) return MAXE_ERR_OOM;
  b->capacity = capacity;
  b->al = Allocator(alloc, st);
  b->sms = di.sms;
  b->status = di.status;
  // one table slot per item plus a sentinel, for each (value type, kernel class)
  const size_t ni = static_cast<size_t>(capacity) * 3 * kClasses, nt = static_cast<size_t>(capacity + 1) * 3 * kClasses;
  if (cudaMallocHost(reinterpret_cast<void**>(&b->h_items), ni * sizeof(BatchItem)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->h_task0), nt * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    batch_release(b);
    return MAXE_ERR_OOM;
  }
  b->d_items = static_cast<BatchItem*>(b->al.get(ni * sizeof(BatchItem)));
  b->d_task0 = static_cast<int32_t*>(b->al.get(nt * sizeof(int32_t)));
  b->d_next = static_cast<int32_t*>(b->al.get(3 * kClasses * sizeof(int32_t)));
  if (!b->d_items || !b->d_task0 || !b->d_next) {
    batch_release(b);
    return MAXE_ERR_OOM;
  }
  if (cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    b->uploaded = nullptr;
    batch_release(b);
    return MAXE_ERR_CUDA;
  }
  b->items.reserve(capacity);
  *out = b;
  return MAXE_OK;
}

maxe_status maxe_batch_set(maxe_batch* b, const maxe_batch_item* items, int32_t n) {
  if (!b || n < 0 || n > b->capacity || (n > 0 && !items)) return MAXE_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i) {
    const maxe_batch_item& a = items[i];
    if (!a.h || a.k < 1 || a.k > 64 || a.ldx < a.k || a.ldy < a.k) return MAXE_ERR_INVALID;
    if ((a.h->cols > 0 && !a.X) || (a.h->rows > 0 && !a.Y)) return MAXE_ERR_INVALID;
    if (a.flags & ~static_cast<uint32_t>(MAXE_BATCH_SCATTER_Y)) return MAXE_ERR_INVALID;
    if (!a.h->bwrow) return MAXE_ERR_INVALID;
  }
  b->items.assign(items, items + n);
  b->n = n;
  return MAXE_OK;
}

maxe_status maxe_batch_run(maxe_batch* b, void* stream) {
  if (!b) return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MAXE_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  // the staging is read by the previous run's copies when they execute: wait for them
  if (b->pending && cap == cudaStreamCaptureStatusNone) {
    MAXE_CUDA_TRY(cudaEventSynchronize(b->uploaded));
    b->pending = false;
  }
  // items without nonzeros: Y = 0, written here; no kernel reads their X
  for (const maxe_batch_item& a : b->items) {
    const maxe_handle* h = a.h;
    if (h->rows == 0 || h->nnz > 0) continue;
    const size_t eb = static_cast<size_t>(vector_bytes(h->dtype));
    MAXE_CUDA_TRY(cudaMemset2DAsync(a.Y, static_cast<size_t>(a.ldy) * eb, 0, static_cast<size_t>(a.k) * eb,
                                    static_cast<size_t>(h->rows), st));
  }
  const maxe_dtype types[3] = {MAXE_F64, MAXE_F32, MAXE_BF16};
  for (int g = 0; g < 3 * kClasses; ++g) {
    const int ti = g / kClasses, cls = g % kClasses;
    BatchItem* hi = b->h_items + static_cast<size_t>(g) * b->capacity;
    int32_t* ht = b->h_task0 + static_cast<size_t>(g) * (b->capacity + 1);
    int32_t m = 0;
    int64_t tasks = 0;
    int bps = 0;  // the largest CTA count per SM the items' plans ask for (0: as many as fit)
    bool any_default = false;
    for (const maxe_batch_item& a : b->items) {
      const maxe_handle* h = a.h;
      if (h->dtype != types[ti] || h->rows == 0 || h->nnz == 0) continue;
      const int eb = vector_bytes(h->dtype);
      const int vw = pick_vw(a, eb);
      const int unit = (a.k == 1 && a.ldx == 1 && a.ldy == 1) ? 1 : 0;
      const int it16 = (unit && h->bit16) ? 1 : 0;
      const bool rows = !unit && h->blc == 2 && spmm_rows_ready(h, a.k, a.X, a.ldx, a.Y, a.ldy);
      if (item_class(vw, unit, it16, rows) != cls) continue;
      BatchItem& d = hi[m];
      d.rowptr = h->rowptr;
      d.col = h->col;
      d.val = h->val;
      d.X = a.X;
      d.Y = a.Y;
      d.yperm = (a.flags & MAXE_BATCH_SCATTER_Y) ? h->rperm : nullptr;
      d.wrow = h->bwrow;
      d.ldx = a.ldx;
      d.ldy = a.ldy;
      d.k = a.k;
      d.M = h->rows;
      d.nW = h->bnW;
      d.vw = vw;
      d.unit = unit;
      d.it16 = it16;
      d.lcg = (unit || h->blc != 1) ? 0 : lc_group(a.k, eb, static_cast<int>(a.ldx % 1024), static_cast<int>(a.ldy % 1024));
      if (d.lcg > 0 && vw < (eb == 4 ? 4 : 2)) d.lcg = 0;  // needs 16-byte aligned X and Y rows
      ht[m] = static_cast<int32_t>(tasks);
      tasks += h->bnW;
      ++m;
      if (h->bbps == 0)
        any_default = true;
      else
        bps = std::max(bps, h->bbps);
    }
    if (any_default) bps = 0;
    if (m == 0) continue;
    if (tasks > INT32_MAX) return MAXE_ERR_UNSUPPORTED;
    ht[m] = static_cast<int32_t>(tasks);
    BatchItem* di = b->d_items + static_cast<size_t>(g) * b->capacity;
    int32_t* dt = b->d_task0 + static_cast<size_t>(g) * (b->capacity + 1);
    MAXE_CUDA_TRY(cudaMemcpyAsync(di, hi, sizeof(BatchItem) * m, cudaMemcpyHostToDevice, st));
    MAXE_CUDA_TRY(cudaMemcpyAsync(dt, ht, sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice, st));
    MAXE_CUDA_TRY(cudaMemsetAsync(b->d_next + g, 0, sizeof(int32_t), st));
    BatchParams bp{di, dt, b->status, b->d_next + g, m, static_cast<int32_t>(tasks), wait_limit_ns()};
    MAXE_TRY(launch_for(types[ti], cls, bp, b->sms, bps, st));
  }
  if (cap == cudaStreamCaptureStatusNone) {
    MAXE_CUDA_TRY(cudaEventRecord(b->uploaded, st));
    b->pending = true;
  }
  return MAXE_OK;
}

maxe_status maxe_batch_destroy(maxe_batch* b) {
  batch_release(b);
  return MAXE_OK;
}

maxe_status maxe_batch_tune(maxe_handle* h, int32_t k, void* stream) {
  if (!h || k < 1 || k > 64) return MAXE_ERR_INVALID;
  if (h->rows == 0 || h->nnz == 0) return MAXE_OK;
  cudaStream_t st = as_stream(stream);
  const int eb = vector_bytes(h->dtype);
  // rows padded to whole vectors, as callers are advised to lay X and Y out
  const int32_t kp = k == 1 ? 1 : static_cast<int32_t>(round_up(k, eb == 4 ? 4 : 2));
  ScratchSet scratch(h->al);
  void* X = scratch.get<unsigned char>(static_cast<size_t>(h->cols) * kp * eb);
  void* Y = scratch.get<unsigned char>(static_cast<size_t>(h->rows) * kp * eb);
  if (!X || !Y) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemsetAsync(X, 0, static_cast<size_t>(h->cols) * kp * eb, st));
  constexpr int kMaxCopies = 64;
  maxe_batch* b = nullptr;
  MAXE_TRY(maxe_batch_create(kMaxCopies, nullptr, stream, &b));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  maxe_status s = (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) ? MAXE_OK
                                                                                             : MAXE_ERR_CUDA;
  const int64_t resident = batch_resident_warps(h->dtype, h->sms);
  const int64_t floor_h = ceil_div(h->nnz, resident);
  struct Plan {
    int64_t H;
    int it16, lc, bps;
  };
  // the plan the handle has (the default unless tuned before)
  const Plan current{h->bH, h->bit16, h->blc, h->bbps};
  maxe_batch_item items[kMaxCopies];
  // Throughput, not latency: the matrix is timed as one of many items, so the
  // item is repeated until the current plan's tasks fill the resident warps
  // once and four times over; every plan is timed on the same copies, that is
  // on the same work (the copies write identical values to one Y; only the
  // time is used).  Returns ms per copy, the best of three timings of 3 runs.
  const int64_t copies1 = std::max<int64_t>(1, std::min<int64_t>(kMaxCopies, ceil_div(resident, h->bnW)));
  const int64_t copies4 = std::max<int64_t>(1, std::min<int64_t>(kMaxCopies, ceil_div(4 * resident, h->bnW)));
  auto time_fill = [&](int fill, float* per_copy) -> maxe_status {
    const int64_t copies = fill == 1 ? copies1 : copies4;
    for (int64_t c = 0; c < copies; ++c) items[c] = maxe_batch_item{h, k, X, kp, Y, kp, 0u};
    MAXE_TRY(maxe_batch_set(b, items, static_cast<int32_t>(copies)));
    for (int rep = 0; rep < 2; ++rep) MAXE_TRY(maxe_batch_run(b, stream));
    float best = 1e30f;
    for (int trial = 0; trial < 3; ++trial) {
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3; ++rep) MAXE_TRY(maxe_batch_run(b, stream));
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return MAXE_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms / static_cast<float>(copies));
    }
    *per_copy = best;
    return MAXE_OK;
  };
  // A plan is timed in a batch that fills the GPU about once (where large
  // tasks leave a tail) and four times over (where they do not).
  auto time_plan = [&](const Plan& pl, float* t1, float* t4) -> maxe_status {
    MAXE_TRY(batch_plan(h, pl.H, pl.it16, st, pl.lc, pl.bps));
    MAXE_TRY(time_fill(1, t1));
    return time_fill(4, t4);
  };
  float c1 = 1e30f, c4 = 1e30f;
  if (s == MAXE_OK) s = time_plan(current, &c1, &c4);
  // a candidate's score: its slower side relative to the current plan
  auto score = [&](float t1, float t4) { return std::max(t1 / c1, t4 / c4); };
  Plan best = current;
  float t_best = 1.0f;  // the current plan's score
  const float t_current = 1.0f;
  // 1) entries per task and the kernel variant, at the launch's full CTA count
  const int64_t cand_h[4] = {std::max<int64_t>(512, floor_h), std::max<int64_t>(2048, floor_h),
                             std::max<int64_t>(8192, floor_h), std::max<int64_t>(32768, floor_h)};
  for (int ci = 0; ci < 4 && s == MAXE_OK; ++ci) {
    if (ci > 0 && cand_h[ci] == cand_h[ci - 1]) continue;
    for (int var = 0; var <= (k == 1 ? 1 : 2) && s == MAXE_OK; ++var) {
      // k = 1: 8 or 16 entries per lane; k > 1: column passes, columns across
      // lanes, one row per lane group
      const Plan pl{cand_h[ci], (k == 1) ? var : 0, (k > 1) ? var : 0, 0};
      if (var == 1 && k > 1 && lc_group(k, eb, kp % 1024, kp % 1024) == 0) continue;
      if (var == 2 && !spmm_rows_ready(h, k, X, kp, Y, kp)) continue;
      if (pl.H == current.H && pl.it16 == current.it16 && pl.lc == current.lc && pl.bps == current.bps) continue;
      float t1 = 0.f, t4 = 0.f;
      s = time_plan(pl, &t1, &t4);
      if (s == MAXE_OK && score(t1, t4) < t_best) {
        t_best = score(t1, t4);
        best = pl;
      }
    }
  }
  // 2) CTAs per SM (the CTA shape of the launch) for the best of those
  const int cls = (k == 1) ? (best.it16 ? 1 : 0) : (best.lc == 2 ? 3 : 2);
  const int occ = batch_occupancy(h->dtype, cls);
  const Plan base = best;
  for (int bps = occ - 1; bps >= 1 && s == MAXE_OK; --bps) {
    Plan pl = base;
    pl.bps = bps;
    float t1 = 0.f, t4 = 0.f;
    s = time_plan(pl, &t1, &t4);
    if (s == MAXE_OK && score(t1, t4) < t_best) {
      t_best = score(t1, t4);
      best = pl;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  maxe_batch_destroy(b);
  // the handle's plan stays unless a candidate was at least 3% faster at both fills
  if (t_best > 0.97f * t_current) best = current;
  if (s == MAXE_OK) s = batch_plan(h, best.H, best.it16, st, best.lc, best.bps);
  if (s == MAXE_OK && cudaStreamSynchronize(st) != cudaSuccess) s = MAXE_ERR_CUDA;
  return s;
}

maxe_status maxe_batch_plan_shape(const maxe_handle* h, int32_t* blocks_per_sm) {
  if (!h || !blocks_per_sm) return MAXE_ERR_INVALID;
  *blocks_per_sm = h->bbps;
  return MAXE_OK;
}

maxe_status maxe_batch_plan_info(const maxe_handle* h, int64_t* entries_per_task, int32_t* tasks,
                                 int32_t* items_per_lane) {
  if (!h) return MAXE_ERR_INVALID;
  if (entries_per_task) *entries_per_task = h->bH;
  if (tasks) *tasks = h->bnW;
  if (items_per_lane) *items_per_lane = h->bit16 ? 16 : 8;
  return MAXE_OK;
}

}  // extern "C"
