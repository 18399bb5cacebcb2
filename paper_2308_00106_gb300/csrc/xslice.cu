// xslice.cu -- SpMV with x staged in shared memory by column slices.
//
// On a randomly permuted matrix every nonzero of the CSR kernel gathers x[col]
// from a random address: one L2 request per nonzero, which bounds the product
// well below HBM bandwidth.  Here the columns are cut into slices of S = 2^14
// (FP32) / 2^13 (FP64) columns, 64 KB of x each, and the matrix into tiles of
// consecutive rows, one tile per SM at a time:
//
//   - a producer warp loads the slices of x the tile touches, in order, into a
//     shared-memory ring of three (FP64: two) slices with 1-D bulk copies (TMA;
//     64 KB, L2 evict-last so x stays in L2 for the other SMs);
//   - 15 consumer warps each own a contiguous range of the tile's rows
//     (nnz-balanced) and a row accumulator per row in shared memory; the
//     entries of one warp range and one slice (a cell, in row order) are cut
//     into 32 contiguous runs of equal length, one per lane, and stored step by
//     step (entry j of every lane's run side by side), so a warp reads a cell
//     with one coalesced 128-byte load per step and no lane idles;
//   - every entry adds a * x[col] to its row's accumulator.  A row that a lane
//     boundary cuts is split: the entries before the cut go to the lane's own
//     scratch accumulator, the ones after it to the row, and after the cell the
//     lane that holds the row's last run reads the scratch sums of the lanes
//     the row came through from shared memory and adds them to the row;
//   - two register groups of 8 steps per warp, one summed while the other
//     loads; with large cells a second cursor prefetches the entries four
//     groups ahead into L2;
//   - at the end of the tile every warp writes its rows of y (through rperm
//     when y is wanted in the original space).
//
// Within a cell every accumulator has one writer lane, across cells the order
// is slice order, and the scratch sums are combined in lane order, so the
// result is deterministic.  The format is built once from the handle's CSR (a
// stable sort by (warp range, slice)); it pays when the rows of a tile hit most
// x sectors of the slices they touch, i.e. for matrices with many nonzeros per
// column of a tile (the 1M-row power-law matrix permuted), and unless asked
// for explicitly it is skipped when the estimated x traffic exceeds four times
// the matrix.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kXsWarps = 15;  // consumer warps per CTA; with the producer, 4 warps per SM sub-partition
constexpr int kXsThreads = 32 * (kXsWarps + 1);
constexpr int kXsSteps = 8;     // steps of a cell per register group
constexpr int kXsAlign = 32;    // cell starts padded to 32 entries: each step is one aligned run of 32
constexpr int kXsSlack = 256;   // zeroed entries after the last cell
constexpr int kXsColBits = 15;  // idx = (accumulator << 15) | column in slice; column S is a zero
constexpr uint32_t kXsColMask = (1u << kXsColBits) - 1u;

template <typename VT>
struct XsCfg;
template <>
struct XsCfg<float> {
  static constexpr int kSliceBits = 14;  // 16384 columns, 64 KB
  static constexpr int kBuffers = 3;     // slices in the ring: two loads in flight while one is read
  static constexpr int kRows = 8192;     // rows per tile
};
template <>
struct XsCfg<double> {
  static constexpr int kSliceBits = 13;  // 8192 columns, 64 KB
  static constexpr int kBuffers = 2;
  static constexpr int kRows = 8192;
};

// One slot of the ring: the slice and 16 bytes after it, the first element of
// which stays zero (the column of the entries a lane pads its run with).
template <typename VT>
constexpr int xs_slot_elems() {
  return (1 << XsCfg<VT>::kSliceBits) + 16 / static_cast<int>(sizeof(VT));
}

// Accumulators: kRows rows of the tile, then 32 scratch sums per consumer warp.
template <typename VT>
constexpr int xs_acc_elems() {
  return XsCfg<VT>::kRows + 32 * kXsWarps;
}

template <typename VT>
constexpr size_t xs_smem_bytes() {
  return sizeof(VT) * (XsCfg<VT>::kBuffers * static_cast<size_t>(xs_slot_elems<VT>()) + xs_acc_elems<VT>()) +
         16 * XsCfg<VT>::kBuffers + 16;
}

struct XsParams {
  const uint32_t* idx;        // (accumulator << 15) | column in slice, cell by cell, step-major
  const void* val;            // values, aligned with idx
  const int32_t* seg_start;   // [G * nS] first slot of (warp range, slice)
  const int32_t* seg_len;     // [G * nS] entries of (warp range, slice)
  const uint32_t* seg_cut;    // [G * nS] bit l: the last row of lane l's run continues in lane l + 1
  const int32_t* tile_row;    // [ntiles + 1]
  const int32_t* warp_row;    // [G + 1] first (global) row of each warp range
  const int32_t* tl_off;      // [ntiles + 1] into tl_slice
  const int32_t* tl_slice;    // slices touched by each tile, ascending
  int32_t ntiles, nS, N;
  const void* x;
  void* y;
  const int32_t* yperm;
  unsigned* status;
};

// Prefetch `bytes` at p (16-byte aligned, a multiple of 16) into L2; no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

template <typename ValT>
struct XsVal;
template <>
struct XsVal<double> {  // FP64 values
  using AT = double;
  static __device__ __forceinline__ double ld(const void* v, int64_t e) {
    return __ldcs(static_cast<const double*>(v) + e);
  }
};
template <>
struct XsVal<float> {  // FP32 values
  using AT = float;
  static __device__ __forceinline__ float ld(const void* v, int64_t e) {
    return __ldcs(static_cast<const float*>(v) + e);
  }
};
template <>
struct XsVal<uint16_t> {  // BF16 values, FP32 arithmetic
  using AT = float;
  static __device__ __forceinline__ float ld(const void* v, int64_t e) {
    return __uint_as_float(static_cast<uint32_t>(__ldcs(static_cast<const unsigned short*>(v) + e)) << 16);
  }
};

// A group of up to kXsSteps consecutive steps of a lane's run, in registers.
template <typename AT>
struct XsGroup {
  uint32_t id[kXsSteps];
  AT a[kXsSteps];
};

// Position of a group in a warp's stream over the tile's slices: slice index i
// (into tl_slice), the cell (n entries in the 32 * ceil(n / 32) slots from
// slot st) with its cut mask, and the first step s0 of the group; i = -1 past
// the end.  The cells of 32 slices at a time sit
// in the lanes (lane l: slice index base + l), so finding the next slice with
// entries is a ballot.
struct XsPos {
  int i;
  int32_t st, n, s0;
  uint32_t cut;
};

struct XsWindow {
  int base;  // slice index held by lane 0
  int32_t st, n;
  uint32_t cut;
};

__device__ __forceinline__ void xs_window_load(const XsParams& p, int64_t g, int i_end, int base, int lane,
                                               XsWindow& w) {
  w.base = base;
  const int i = base + lane;
  if (i < i_end) {
    const int64_t key = g * p.nS + p.tl_slice[i];
    w.st = p.seg_start[key];
    w.n = p.seg_len[key];
    w.cut = p.seg_cut[key];
  } else {
    w.st = 0;
    w.n = 0;
    w.cut = 0;
  }
}

// The first group of the first slice index > i with entries of this warp.
__device__ __forceinline__ XsPos xs_next_slice(const XsParams& p, int64_t g, int i, int i_end, int lane,
                                               XsWindow& w) {
  while (true) {
    const int li = w.base + lane;
    const unsigned m = __ballot_sync(0xffffffffu, li > i && li < i_end && w.n > 0);
    if (m) {
      const int src = __ffs(m) - 1;
      XsPos q;
      q.i = w.base + src;
      q.st = __shfl_sync(0xffffffffu, w.st, src);
      q.n = __shfl_sync(0xffffffffu, w.n, src);
      q.cut = __shfl_sync(0xffffffffu, w.cut, src);
      q.s0 = 0;
      return q;
    }
    if (w.base + 32 >= i_end) return XsPos{-1, 0, 0, 0, 0u};
    xs_window_load(p, g, i_end, w.base + 32, lane, w);
  }
}

__device__ __forceinline__ int32_t xs_steps(int32_t n) { return (n + 31) >> 5; }

__device__ __forceinline__ XsPos xs_next(const XsParams& p, int64_t g, const XsPos& q, int i_end, int lane,
                                         XsWindow& w) {
  if (q.i < 0) return q;
  if (q.s0 + kXsSteps < xs_steps(q.n)) return XsPos{q.i, q.st, q.n, q.s0 + kXsSteps, q.cut};
  return xs_next_slice(p, g, q.i, i_end, lane, w);
}

// Load the group's steps (those of the cell's L steps) of this lane's run.
// The slots past a lane's run hold a pad entry (the lane's scratch sum, the
// zero column, value 0), so every lane loads every step unconditionally.
template <typename ValT>
__device__ __forceinline__ void xs_load(const XsParams& p, const XsPos& q, int lane,
                                        XsGroup<typename XsVal<ValT>::AT>& k) {
  const int32_t ns = xs_steps(q.n) - q.s0;
  const int64_t base = static_cast<int64_t>(q.st) + static_cast<int64_t>(q.s0) * 32 + lane;
#pragma unroll
  for (int j = 0; j < kXsSteps; ++j) {
    if (j < ns) {
      k.id[j] = __ldcs(p.idx + base + 32 * j);
      k.a[j] = XsVal<ValT>::ld(p.val, base + 32 * j);
    }
  }
}

// With large cells (the entries of a warp in a slice span several groups) a
// second cursor runs kXsAhead groups ahead of the loads and prefetches their
// entries into L2, so the loads find them there; with small cells its
// bookkeeping per group costs more than it hides.
constexpr int kXsAhead = 4;
constexpr int64_t kXsPrefetchCell = 2 * 32 * kXsSteps;  // mean entries per cell from which the cursor runs

template <typename ValT>
__device__ __forceinline__ void xs_prefetch(const XsParams& p, const XsPos& q, int lane) {
  if (q.i < 0 || lane != 0) return;
  const int32_t L = xs_steps(q.n);
  const int32_t ns = L - q.s0 < kXsSteps ? L - q.s0 : kXsSteps;
  const int64_t base = static_cast<int64_t>(q.st) + static_cast<int64_t>(q.s0) * 32;
  prefetch_l2(p.idx + base, static_cast<uint32_t>(ns * 32 * 4));
  prefetch_l2(static_cast<const unsigned char*>(p.val) + base * static_cast<int64_t>(sizeof(ValT)),
              static_cast<uint32_t>(ns * 32 * sizeof(ValT)));
}

// acc[slot] += a * x[column] for the group's first ns steps.
template <typename VT, typename AT>
__device__ __forceinline__ void xs_compute(const XsGroup<AT>& k, int ns, const VT* __restrict__ xs,
                                           VT* __restrict__ acc) {
#pragma unroll
  for (int j = 0; j < kXsSteps; ++j) {
    if (j < ns) {
      const uint32_t u = k.id[j];
      const VT xv = xs[u & kXsColMask];
      VT* ap = acc + (u >> kXsColBits);
      *ap = fma(static_cast<VT>(k.a[j]), xv, *ap);
    }
  }
}

// After a cell: add the scratch sums of the rows cut by lane boundaries to the
// rows.  cut bit l: lane l's last row continues in lane l + 1 (its entries of
// that row went to scratch[l]).  f0: the accumulator of the lane's first
// entry -- a row, or the lane's scratch when the lane's first row continues
// (then the lane holds that row only and the row runs through it).  The lane
// whose first row came from the previous lane and ends in it reads the
// chain's scratch sums from shared memory, last lane first, and adds them to
// the row; then the lanes clear their scratch sums.
template <typename VT>
__device__ __forceinline__ void xs_combine(uint32_t cut, uint32_t f0, VT* __restrict__ acc,
                                           VT* __restrict__ scratch, int lane) {
  constexpr uint32_t kRows = XsCfg<VT>::kRows;
  const bool in = lane > 0 && ((cut >> (lane - 1)) & 1u);
  const bool through = in && f0 >= kRows;
  const unsigned thr = __ballot_sync(0xffffffffu, through);
  __syncwarp();  // every lane's scratch sum is written
  if (in && !through) {
    VT sum = VT(0);
    for (int m = lane - 1;; --m) {  // ends at the chain's first lane (not run through; lane 0 never is)
      sum += scratch[m];
      if (!((thr >> m) & 1u)) break;
    }
    acc[f0] += sum;
  }
  __syncwarp();  // read before cleared
  if ((cut >> lane) & 1u) scratch[lane] = VT(0);
}

template <typename VT, typename ValT, bool PF>
__global__ void __launch_bounds__(kXsThreads, 1) spmv_xslice_kernel(const XsParams p) {
  using AT = typename XsVal<ValT>::AT;
  constexpr int S = 1 << XsCfg<VT>::kSliceBits;
  constexpr int kSlot = xs_slot_elems<VT>();
  constexpr int NX = XsCfg<VT>::kBuffers;
  constexpr uint32_t kRows = XsCfg<VT>::kRows;
  extern __shared__ __align__(128) unsigned char smem[];
  VT* xb = reinterpret_cast<VT*>(smem);  // [NX][kSlot]
  VT* acc = xb + NX * kSlot;             // [kRows + 32 * kXsWarps]
  uint64_t* full = reinterpret_cast<uint64_t*>(acc + xs_acc_elems<VT>());
  uint64_t* empty = full + NX;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < NX) xb[threadIdx.x * kSlot + S] = VT(0);  // the zero column of each slot
  if (threadIdx.x == 0) {
    for (int b = 0; b < NX; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], kXsWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kXsWarps) {  // ---------------------------------------- producer
    if (lane != 0) return;
    const uint64_t pol = policy_evict_last();
    uint32_t v = 0;
    bool ok = true;
    for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x) {
      for (int i = p.tl_off[t]; i < p.tl_off[t + 1]; ++i, ++v) {
        const int b = v % NX;
        if (v >= NX && !mbar_wait_bounded(&empty[b], (v / NX - 1) & 1u, p.status)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        if (*abort_flag) {
          ok = false;
          break;
        }
        const int64_t c0 = static_cast<int64_t>(p.tl_slice[i]) << XsCfg<VT>::kSliceBits;
        const int width = static_cast<int>((p.N - c0 < S ? p.N - c0 : static_cast<int64_t>(S)));
        constexpr int kVec = 16 / sizeof(VT);
        const int wb = width / kVec * kVec;  // by bulk copy; the rest (< 16 bytes) by this thread
        VT* dst = xb + b * kSlot;
        const VT* src = static_cast<const VT*>(p.x) + c0;
        if (wb < width) {
          for (int k = wb; k < width; ++k) dst[k] = src[k];
          fence_proxy_async_smem();  // a later bulk copy may overwrite these addresses
        }
        mbar_arrive_expect_tx(&full[b], static_cast<uint32_t>(wb * sizeof(VT)));
        if (wb > 0) bulk_g2s(dst, src, static_cast<uint32_t>(wb * sizeof(VT)), &full[b], pol);
      }
    }
    // copies still in flight land before the block can exit
    for (uint32_t u = v > NX ? v - NX : 0; u < v; ++u) mbar_wait_bounded(&full[u % NX], (u / NX) & 1u, p.status);
    return;
  }

  // ------------------------------------------------------------- consumers
  // Each warp keeps two groups in registers: while one is summed, the other
  // is in flight, across slice boundaries (a warp often has one group per
  // slice).  Slice i's buffer is waited for before its first group is
  // summed and released after its last; slices without entries of this warp
  // are waited for and released in turn, so every warp arrives once per slice.
  VT* y = static_cast<VT*>(p.y);
  VT* scratch = acc + kRows + 32 * warp;
  uint32_t v = 0;  // slices visited by this CTA, as counted by the producer
  bool ok = true;
  for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    const int32_t tr0 = p.tile_row[t];
    const int64_t g = static_cast<int64_t>(t) * kXsWarps + warp;
    const int32_t r_lo = p.warp_row[g] - tr0, r_hi = p.warp_row[g + 1] - tr0;
    const int i0 = p.tl_off[t], i1 = p.tl_off[t + 1];
    for (int32_t r = r_lo + lane; r < r_hi; r += 32) acc[r] = VT(0);
    scratch[lane] = VT(0);
    __syncwarp();
    XsWindow win;
    xs_window_load(p, g, i1, i0, lane, win);
    // Two register groups with fixed roles, A and B, summed in turn: while one
    // is summed the other's loads are in flight.  (Rotating one array of
    // groups would copy registers whose loads are still in flight, and the
    // copy waits for them.)
    XsGroup<AT> kA, kB;
    XsPos qA = xs_next_slice(p, g, i0 - 1, i1, lane, win);
    XsPos qB = xs_next(p, g, qA, i1, lane, win);
    if (qA.i >= 0) xs_load<ValT>(p, qA, lane, kA);
    if (qB.i >= 0) xs_load<ValT>(p, qB, lane, kB);
    XsPos qn = xs_next(p, g, qB, i1, lane, win);  // the group after the two in registers
    XsWindow winp;  // the prefetch cursor, kXsAhead groups ahead of the loads (PF)
    XsPos qp{-1, 0, 0, 0, 0u};
    if constexpr (PF) {
      xs_window_load(p, g, i1, i0, lane, winp);
      qp = xs_next_slice(p, g, i0 - 1, i1, lane, winp);
      for (int d = 0; d < 2 + kXsAhead; ++d) {
        if (d >= 2) xs_prefetch<ValT>(p, qp, lane);
        qp = xs_next(p, g, qp, i1, lane, winp);
      }
    }
    int i = i0;         // next slice to wait for
    bool held = false;  // slice i - 1 is waited for and not yet released
    uint32_t f0 = 0;    // accumulator of this lane's first entry in the current cell
    auto sum_group = [&](const XsPos& qc, const XsGroup<AT>& grp) {
      while (i <= qc.i) {  // wait for slices up to this group's, releasing the empty ones
        if (held && lane == 0 && ok) mbar_arrive(&empty[(v - 1) % NX]);
        if (ok) {
          ok = mbar_wait_bounded(&full[v % NX], (v / NX) & 1u, p.status);
          ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
          if (!ok) *abort_flag = 1;
        }
        held = true;
        ++i;
        ++v;
      }
      if (ok) {
        const int32_t L = xs_steps(qc.n);
        if (qc.s0 == 0) f0 = grp.id[0] >> kXsColBits;
        xs_compute<VT, AT>(grp, L - qc.s0 < kXsSteps ? L - qc.s0 : kXsSteps, xb + ((v - 1) % NX) * kSlot, acc);
        if (qc.s0 + kXsSteps >= L) {  // the cell's last group
          if (qc.cut) xs_combine<VT>(qc.cut, f0, acc, scratch, lane);
          __syncwarp();  // the next cell may give this cell's rows to other lanes
        }
      }
    };
    while (qA.i >= 0) {
      sum_group(qA, kA);
      qA = qn;
      if (qA.i >= 0) xs_load<ValT>(p, qA, lane, kA);
      qn = xs_next(p, g, qn, i1, lane, win);
      if constexpr (PF) {
        xs_prefetch<ValT>(p, qp, lane);
        qp = xs_next(p, g, qp, i1, lane, winp);
      }
      if (qB.i < 0) break;
      sum_group(qB, kB);
      qB = qn;
      if (qB.i >= 0) xs_load<ValT>(p, qB, lane, kB);
      qn = xs_next(p, g, qn, i1, lane, win);
      if constexpr (PF) {
        xs_prefetch<ValT>(p, qp, lane);
        qp = xs_next(p, g, qp, i1, lane, winp);
      }
    }
    while (i < i1) {  // slices after this warp's last entries
      if (held && lane == 0 && ok) mbar_arrive(&empty[(v - 1) % NX]);
      if (ok) {
        ok = mbar_wait_bounded(&full[v % NX], (v / NX) & 1u, p.status);
        ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
        if (!ok) *abort_flag = 1;
      }
      held = true;
      ++i;
      ++v;
    }
    if (held && lane == 0 && ok) mbar_arrive(&empty[(v - 1) % NX]);
    __syncwarp();
    if (ok)
      for (int32_t r = r_lo + lane; r < r_hi; r += 32) {
        const int32_t row = tr0 + r;
        y[p.yperm ? p.yperm[row] : row] = acc[r];
      }
    named_bar(1, 32 * kXsWarps);  // the next tile re-partitions the accumulators
  }
}

// ------------------------------------------------------------- building

// keys[e] = (row << 32) | (warp range * nS + slice); counts per (warp range, slice).
__global__ void xs_key_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t M,
                              int64_t Z, const int32_t* __restrict__ warp_row, int32_t G, int32_t nS, int sbits,
                              uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int32_t* __restrict__ counts) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= Z) return;
  int32_t lo = 0, hi = M;  // row: last i with rowptr[i] <= e
  while (hi - lo > 1) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (rowptr[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  int32_t glo = 0, ghi = G;  // warp range: last g with warp_row[g] <= row
  while (ghi - glo > 1) {
    const int32_t mid = glo + (ghi - glo) / 2;
    if (warp_row[mid] <= lo)
      glo = mid;
    else
      ghi = mid;
  }
  const uint32_t key = static_cast<uint32_t>(glo) * static_cast<uint32_t>(nS) + static_cast<uint32_t>(col[e] >> sbits);
  keys[e] = (static_cast<uint64_t>(static_cast<uint32_t>(lo)) << 32) | key;
  vals[e] = static_cast<int32_t>(e);
  atomicAdd(counts + key, 1);
}

// Place sorted entry i (rank `rank` of n in its cell) in its lane's run: the cell's
// n entries are cut into 32 contiguous runs, the first rem = n - 32 (L - 1) of
// L entries and the rest of L - 1, and run entry j of lane l goes to slot
// seg_start + 32 j + l.  An entry whose row continues in the next lane's run
// accumulates into the lane's scratch sum (kRows + 32 w + l, w the warp range
// within the tile), every other entry into its tile-local row; the lane's last
// entry sets cut bit l when its row continues.
__global__ void xs_scatter_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals, int64_t Z,
                                  const int32_t* __restrict__ seg_start, const int32_t* __restrict__ seg_len,
                                  const int32_t* __restrict__ ustart, const int32_t* __restrict__ col,
                                  const void* __restrict__ val, int vbytes, const int32_t* __restrict__ tile_row,
                                  int sbits, int32_t nS, int32_t rows_per_tile, uint32_t* __restrict__ idx_out,
                                  void* __restrict__ val_out, uint32_t* __restrict__ cut_out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Z) return;
  const uint64_t k = keys[i];
  const uint32_t key = static_cast<uint32_t>(k);
  const int32_t row = static_cast<int32_t>(k >> 32);
  const int32_t e = vals[i];
  const int32_t g = static_cast<int32_t>(key / static_cast<uint32_t>(nS));
  const int32_t t = g / kXsWarps, w = g % kXsWarps;
  const int32_t first = ustart[key];
  const int32_t rank = static_cast<int32_t>(i - first), n = seg_len[key];
  const int32_t L = (n + 31) / 32, rem = n - 32 * (L - 1);
  int32_t l, j;
  if (rank < rem * L) {
    l = rank / L;
    j = rank % L;
  } else {  // L >= 2 here
    l = rem + (rank - rem * L) / (L - 1);
    j = (rank - rem * L) % (L - 1);
  }
  const int32_t next = l * (L - 1) + (l < rem ? l : rem) + (l < rem ? L : L - 1);  // first rank of lane l + 1
  const bool crosses = next < n && static_cast<int32_t>(keys[first + next] >> 32) == row;
  const uint32_t acc = crosses ? static_cast<uint32_t>(rows_per_tile + 32 * w + l)
                               : static_cast<uint32_t>(row - tile_row[t]);
  const int64_t pos = static_cast<int64_t>(seg_start[key]) + 32 * static_cast<int64_t>(j) + l;
  idx_out[pos] = (acc << kXsColBits) | (static_cast<uint32_t>(col[e]) & ((1u << sbits) - 1u));
  if (vbytes == 8)
    static_cast<double*>(val_out)[pos] = static_cast<const double*>(val)[e];
  else if (vbytes == 4)
    static_cast<float*>(val_out)[pos] = static_cast<const float*>(val)[e];
  else
    static_cast<uint16_t*>(val_out)[pos] = static_cast<const uint16_t*>(val)[e];
  if (crosses && rank == next - 1) atomicOr(cut_out + key, 1u << l);
  if (rank == n - 1)  // the last step's slots past the runs: pad entries (value 0, zeroed before)
    for (int32_t q = rem; q < 32; ++q)
      idx_out[static_cast<int64_t>(seg_start[key]) + 32 * static_cast<int64_t>(L - 1) + q] =
          (static_cast<uint32_t>(rows_per_tile + 32 * w + q) << kXsColBits) | (1u << sbits);
}

int bit_width_u64(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

template <typename VT, typename ValT>
maxe_status xs_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st) {
  static bool attr_set[64] = {};
  if (h->device >= 0 && h->device < 64 && !attr_set[h->device]) {
    MAXE_CUDA_TRY(cudaFuncSetAttribute(spmv_xslice_kernel<VT, ValT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(xs_smem_bytes<VT>())));
    MAXE_CUDA_TRY(cudaFuncSetAttribute(spmv_xslice_kernel<VT, ValT, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(xs_smem_bytes<VT>())));
    attr_set[h->device] = true;
  }
  XsParams p{};
  p.idx = h->xs_idx;
  p.val = h->xs_val;
  p.seg_start = h->xs_seg_start;
  p.seg_len = h->xs_seg_len;
  p.seg_cut = h->xs_seg_cut;
  p.tile_row = h->xs_tile_row;
  p.warp_row = h->xs_warp_row;
  p.tl_off = h->xs_tl_off;
  p.tl_slice = h->xs_tl_slice;
  p.ntiles = h->xs_ntiles;
  p.nS = h->xs_nS;
  p.N = h->cols;
  p.x = x;
  p.y = y;
  p.yperm = yperm;
  p.status = h->status;
  const int grid = std::min(h->xs_ntiles, h->sms);
  if (h->xs_prefetch)
    spmv_xslice_kernel<VT, ValT, true><<<grid, kXsThreads, xs_smem_bytes<VT>(), st>>>(p);
  else
    spmv_xslice_kernel<VT, ValT, false><<<grid, kXsThreads, xs_smem_bytes<VT>(), st>>>(p);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status build(maxe_handle* h, cudaStream_t st, bool force, bool* built) {
  constexpr int SB = XsCfg<VT>::kSliceBits;
  constexpr int RMAX = XsCfg<VT>::kRows;
  *built = false;
  const int32_t M = h->rows, N = h->cols;
  const int64_t Z = h->nnz;
  if (M == 0 || N == 0 || Z == 0) return MAXE_OK;
  const int vb = value_bytes(h->dtype);
  // ---- tiles and warp ranges, on the host from rowptr
  std::vector<int32_t> rp(static_cast<size_t>(M) + 1);
  MAXE_CUDA_TRY(cudaMemcpyAsync(rp.data(), h->rowptr, sizeof(int32_t) * (M + 1), cudaMemcpyDeviceToHost, st));
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t Ht = std::max<int64_t>(1, ceil_div(Z, std::max(h->sms, 1)));
  std::vector<int32_t> trow{0}, wrow;
  for (int32_t r = 0; r < M;) {
    const int64_t target = rp[r] + Ht;
    int32_t r2 = static_cast<int32_t>(std::lower_bound(rp.begin() + r + 1, rp.end(), target) - rp.begin());
    r2 = std::min<int64_t>({static_cast<int64_t>(r2), static_cast<int64_t>(r) + RMAX, static_cast<int64_t>(M)});
    r2 = std::max(r2, r + 1);
    trow.push_back(r2);
    r = r2;
  }
  const int32_t ntiles = static_cast<int32_t>(trow.size()) - 1;
  for (int32_t t = 0; t < ntiles; ++t) {
    const int32_t a = trow[t], b = trow[t + 1];
    const int64_t E = static_cast<int64_t>(rp[b]) - rp[a];
    int32_t prev = a;
    for (int w = 0; w < kXsWarps; ++w) {
      int32_t r = a;
      if (w > 0) {
        const int64_t target = rp[a] + (E * w + kXsWarps - 1) / kXsWarps;
        r = static_cast<int32_t>(std::lower_bound(rp.begin() + a, rp.begin() + b + 1, target) - rp.begin());
        r = std::min(std::max(r, prev), b);
      }
      wrow.push_back(r);
      prev = r;
    }
  }
  wrow.push_back(M);
  const int64_t G = static_cast<int64_t>(ntiles) * kXsWarps;
  const int32_t nS = static_cast<int32_t>(ceil_div(N, int64_t(1) << SB));
  if (G * nS > (int64_t(1) << 24)) return MAXE_OK;  // too many (warp range, slice) cells to plan
  const int64_t matrix_bytes = Z * (vb + 4);

  const Allocator& al = h->al;
  ScratchSet scratch(al);
  int32_t* d_wrow = static_cast<int32_t*>(al.get(sizeof(int32_t) * (G + 1)));
  int32_t* d_trow = static_cast<int32_t*>(al.get(sizeof(int32_t) * (ntiles + 1)));
  if (!d_wrow || !d_trow) {
    al.put(d_wrow);
    al.put(d_trow);
    return MAXE_ERR_OOM;
  }
  auto fail = [&](maxe_status s) {
    al.put(d_wrow);
    al.put(d_trow);
    return s;
  };
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_wrow, wrow.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_trow, trow.data(), sizeof(int32_t) * (ntiles + 1), cudaMemcpyHostToDevice, st));
  // ---- keys and counts
  const int64_t cells = G * nS;
  uint64_t* keys = scratch.get<uint64_t>(Z);
  uint64_t* keys_alt = scratch.get<uint64_t>(Z);
  int32_t* vals = scratch.get<int32_t>(Z);
  int32_t* vals_alt = scratch.get<int32_t>(Z);
  int32_t* counts = scratch.get<int32_t>(cells);
  void* rs = scratch.get<unsigned char>(radix_scratch_bytes(Z));
  if (!keys || !keys_alt || !vals || !vals_alt || !counts || !rs) return fail(MAXE_ERR_OOM);
  MAXE_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * cells, st));
  xs_key_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(h->rowptr, h->col, M, Z, d_wrow,
                                                                         static_cast<int32_t>(G), nS, SB, keys, vals,
                                                                         counts);
  MAXE_CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> cnt(static_cast<size_t>(cells));
  MAXE_CUDA_TRY(cudaMemcpyAsync(cnt.data(), counts, sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, st));
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  // ---- segment layout, slices per tile, the traffic estimate
  std::vector<int32_t> seg_start(static_cast<size_t>(cells)), ustart(static_cast<size_t>(cells));
  std::vector<int32_t> tl_off{0}, tl_slice;
  int64_t pos = 0, upos = 0;
  for (int64_t k = 0; k < cells; ++k) {
    seg_start[k] = static_cast<int32_t>(pos);
    ustart[k] = static_cast<int32_t>(upos);
    pos += round_up(cnt[k], kXsAlign);
    upos += cnt[k];
  }
  const int64_t Zp = pos;
  if (Zp + kXsSlack > INT32_MAX) return fail(MAXE_OK);
  for (int32_t t = 0; t < ntiles; ++t) {
    for (int32_t s = 0; s < nS; ++s) {
      int64_t any = 0;
      for (int w = 0; w < kXsWarps; ++w) any += cnt[(static_cast<int64_t>(t) * kXsWarps + w) * nS + s];
      if (any) tl_slice.push_back(s);
    }
    tl_off.push_back(static_cast<int32_t>(tl_slice.size()));
  }
  const int64_t x_bytes = static_cast<int64_t>(tl_slice.size()) * sizeof(VT) * (int64_t(1) << SB);
  if (!force && x_bytes > 4 * matrix_bytes) return fail(MAXE_OK);  // the CSR kernel will do better
  // ---- device arrays of the format
  uint32_t* idx = static_cast<uint32_t*>(al.get(sizeof(uint32_t) * (Zp + kXsSlack)));
  void* xval = al.get(static_cast<size_t>(vb) * (Zp + kXsSlack));
  int32_t* d_seg = static_cast<int32_t*>(al.get(sizeof(int32_t) * 3 * cells));
  int32_t* d_ustart = scratch.get<int32_t>(cells);
  int32_t* d_tl = static_cast<int32_t*>(al.get(sizeof(int32_t) * (tl_off.size() + std::max<size_t>(tl_slice.size(), 1))));
  if (!idx || !xval || !d_seg || !d_ustart || !d_tl) {
    al.put(idx);
    al.put(xval);
    al.put(d_seg);
    al.put(d_tl);
    return fail(MAXE_ERR_OOM);
  }
  int32_t* d_len = d_seg + cells;
  uint32_t* d_cut = reinterpret_cast<uint32_t*>(d_seg + 2 * cells);
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_seg, seg_start.data(), sizeof(int32_t) * cells, cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_len, cnt.data(), sizeof(int32_t) * cells, cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_ustart, ustart.data(), sizeof(int32_t) * cells, cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_tl, tl_off.data(), sizeof(int32_t) * tl_off.size(), cudaMemcpyHostToDevice, st));
  if (!tl_slice.empty())
    MAXE_CUDA_TRY(cudaMemcpyAsync(d_tl + tl_off.size(), tl_slice.data(), sizeof(int32_t) * tl_slice.size(),
                                  cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemsetAsync(d_cut, 0, sizeof(uint32_t) * cells, st));
  MAXE_CUDA_TRY(cudaMemsetAsync(idx, 0, sizeof(uint32_t) * (Zp + kXsSlack), st));
  MAXE_CUDA_TRY(cudaMemsetAsync(xval, 0, static_cast<size_t>(vb) * (Zp + kXsSlack), st));
  // ---- stable sort by (warp range, slice); entries keep CSR order inside a cell
  MAXE_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, Z, bit_width_u64(static_cast<uint64_t>(cells - 1)), rs,
                            st));
  xs_scatter_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(
      keys, vals, Z, d_seg, d_len, d_ustart, h->col, h->val, vb, d_trow, SB, nS, RMAX, idx, xval, d_cut);
  MAXE_CUDA_TRY(cudaGetLastError());
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors and scratch go out of scope
  h->xs_idx = idx;
  h->xs_val = xval;
  h->xs_seg_start = d_seg;
  h->xs_seg_len = d_len;
  h->xs_seg_cut = d_cut;
  h->xs_tile_row = d_trow;
  h->xs_warp_row = d_wrow;
  h->xs_tl_off = d_tl;
  h->xs_tl_slice = d_tl + tl_off.size();
  h->xs_ntiles = ntiles;
  h->xs_nS = nS;
  h->xs_bytes = static_cast<int64_t>(Zp) * (4 + vb) + 12 * cells;
  int64_t nonempty = 0;
  for (int64_t k = 0; k < cells; ++k) nonempty += cnt[k] > 0;
  h->xs_prefetch = nonempty > 0 && Z >= kXsPrefetchCell * nonempty ? 1 : 0;
  *built = true;
  return MAXE_OK;
}

}  // namespace

maxe_status xslice_build(maxe_handle* h, cudaStream_t st, bool force) {
  bool built = false;
  maxe_status s = h->dtype == MAXE_F64 ? build<double>(h, st, force, &built) : build<float>(h, st, force, &built);
  if (s == MAXE_OK && built) h->xs_use = 1;
  return s;
}

bool xslice_ready(const maxe_handle* h, const void* x) {
  return h->xs_idx && h->xs_use && (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
}

maxe_status xslice_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st) {
  if (h->dtype == MAXE_F64) return xs_launch<double, double>(h, x, y, yperm, st);
  if (h->dtype == MAXE_F32) return xs_launch<float, float>(h, x, y, yperm, st);
  return xs_launch<float, uint16_t>(h, x, y, yperm, st);
}

void xslice_release(maxe_handle* h) {
  const Allocator& al = h->al;
  al.put(h->xs_tl_off);
  al.put(h->xs_seg_start);
  al.put(h->xs_val);
  al.put(h->xs_idx);
  al.put(h->xs_warp_row);
  al.put(h->xs_tile_row);
  h->xs_tl_off = h->xs_tl_slice = h->xs_seg_start = h->xs_seg_len = nullptr;
  h->xs_seg_cut = nullptr;
  h->xs_warp_row = h->xs_tile_row = nullptr;
  h->xs_idx = nullptr;
  h->xs_val = nullptr;
  h->xs_use = 0;
}

}  // namespace maxe
