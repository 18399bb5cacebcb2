// xslice.cu -- SpMV with x staged in shared memory by column slices.
//
// On a randomly permuted matrix every nonzero of the CSR kernel gathers x[col]
// from a random address: one L2 request per nonzero, which bounds the product
// well below HBM bandwidth.  Here the columns are cut into slices of x that fit
// in shared memory and the rows into tiles, one tile per CTA:
//
//   - a producer warp loads the slices of x the tile touches, in order, into a
//     shared-memory ring (1-D bulk copies through the TMA unit, L2 evict-last so
//     x stays in L2 for the other SMs);
//   - 15 consumer warps each own a contiguous, nnz-balanced range of the tile's
//     rows and an accumulator per row in shared memory.  The entries of one warp
//     range and one slice form a cell; every entry adds a * x[col] to its
//     accumulator;
//   - a cell's n entries go to 32 lane runs of L = ceil(n / 32) or L - 1
//     entries, stored step by step (entry j of every run side by side, the
//     cell starting on a 32-byte sector), so a step is one coalesced load of
//     whole sectors per array.  In cells of at most 32 steps the builder packs
//     each accumulator's entries whole into one run (filling the runs in
//     accumulator order, a group that does not fit the current run going to a
//     later one), so no two lanes of a cell update one accumulator; in longer
//     cells the runs cut the accumulator order where they end, and a cut
//     accumulator is updated by the later lane in its first steps and by the
//     earlier lane in its last steps, at least a register group apart, where
//     the warp synchronises (the rare short cell that cannot be packed is
//     dealt over enough steps for this).  No partial sum leaves its
//     accumulator, so there is nothing to combine;
//   - a row with many entries (more than about 1/96 of its warp's entries) is
//     split into virtual rows, every V-th of its entries in column order, each
//     with an accumulator of its own, so that an accumulator rarely has more
//     entries in a cell than a run is long (a cell where one does is dealt out
//     instead: entry k to lane k / S, step k % S, with S the largest count); a
//     virtual row is added to its row once, at the end of the tile.  Ordering a
//     cell by accumulator bank first spreads the accumulators of a step over the
//     32 shared-memory banks;
//   - optionally (for matrices whose nonzeros spread evenly over the columns,
//     such as a randomly permuted one) the columns are cut in two halves and a
//     tile is run by a cluster of two CTAs, one per half, on two SMs: each SM
//     streams half of x, its cells are twice as large, and at the end each CTA
//     writes half of the tile's rows as its own accumulator plus its partner's,
//     read through distributed shared memory;
//   - with large cells a second cursor prefetches the entries a few groups ahead
//     into L2.
//
// Every accumulator is updated in an order fixed by the format (steps in order,
// cells in slice order, virtual rows in order, the pair's halves in order), so
// the result is deterministic.  The format is built once from the handle's CSR;
// it pays when the rows of a tile hit most x sectors of the slices they touch,
// i.e. for matrices with many nonzeros per column of a tile, and unless asked
// for explicitly it is skipped when the estimated x traffic exceeds eight times
// the matrix.
#include <algorithm>
#include <mutex>
#include <vector>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kXsWarps = 15;  // consumer warps per CTA; with the producer, 4 warps per SM sub-partition
constexpr int kXsThreads = 32 * (kXsWarps + 1);
constexpr int kXsColBits = 15;  // idx = (accumulator << 15) | continues << 14 | column in slice
constexpr uint32_t kXsColMask = (1u << 14) - 1u;  // slices are at most 16384 columns
constexpr uint32_t kXsCont = 1u << 14;  // same accumulator as the lane's previous step in the group
constexpr int kXsSlack = 256;     // zeroed entries after the last cell (L2 prefetches round out to 16 bytes)
constexpr int kXsMaxSlots = 32767;  // accumulators per CTA (the sort key holds 15 bits of accumulator)
constexpr int kXsVirtDiv = 96;    // rows with more than 1/96 of their warp's entries are split
constexpr int kXsVirtMin = 32;    // ... and never into virtual rows shorter than this
constexpr int kXsBarBytes = 128;  // mbarriers and the abort flag at the end of shared memory

// Slice width (columns) and ring depth per vector type and number of column
// halves J.  Steps: steps of a cell per register group.
template <typename VT, int J>
struct XsCfg;
template <>
struct XsCfg<float, 1> {
  static constexpr int kSliceCols = 16384;  // 64 KB
  static constexpr int kBuffers = 3;
  static constexpr int kSteps = 8;
};
template <>
struct XsCfg<float, 2> {
  static constexpr int kSliceCols = 12288;  // 48 KB
  static constexpr int kBuffers = 3;
  static constexpr int kSteps = 10;
};
template <>
struct XsCfg<double, 1> {
  static constexpr int kSliceCols = 8192;  // 64 KB
  static constexpr int kBuffers = 2;
  static constexpr int kSteps = 6;
};

template <typename VT, int J>
constexpr size_t xs_ring_bytes() {
  return sizeof(VT) * static_cast<size_t>(XsCfg<VT, J>::kBuffers) * XsCfg<VT, J>::kSliceCols;
}

// Shared memory of a CTA with `slots` accumulators.
template <typename VT, int J>
size_t xs_smem_bytes(int32_t slots) {
  return xs_ring_bytes<VT, J>() + sizeof(VT) * static_cast<size_t>(slots) + kXsBarBytes;
}

struct XsParams {
  const uint32_t* idx;        // (accumulator << 15) | column in slice, cell by cell, step-major; FP32
                              // values: (index, value bits) pairs
  const void* val;            // other values, aligned with idx (null for FP32)
  const int32_t* seg;         // [3 * cells]: first entry, steps S, layout word (see xs_layout)
  int64_t cells;
  int64_t nent;               // entries allocated in idx and val
  int32_t ahead;              // stream prefetch distance in entries (0: none; see xs_ahead)
  const int32_t* tile_row;    // [ntiles + 1]
  const int32_t* warp_row;    // [ntiles * J * (W + 1)] row ranges of the warps of each (tile, half)
  const int32_t* vslot;       // [ntiles * J * (W + 1)] virtual accumulators of the warps of each (tile, half)
  const int32_t* vl_off;      // [ntiles * J * W + 1] into vl_item
  const int32_t* vl_item;     // [3 * items] split rows: (row accumulator, first virtual accumulator, count)
  const int32_t* tl_off;      // [ntiles * J + 1] into tl_slice
  const int32_t* tl_slice;    // slices touched by each (tile, half), ascending
  int32_t nS, N;
  const void* x;
  void* y;
  const int32_t* yperm;
  unsigned* status;
  uint64_t wait_ns;  // limit of the bounded waits
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

// ---- thread-block cluster of two CTAs (the column halves of a tile)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of both CTAs: writes before it are visible to reads after it in the other CTA.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ float ld_cluster(uint32_t a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

template <typename ValT>
struct XsVal;
template <>
struct XsVal<double> {  // FP64 values
  using AT = double;
  static __device__ __forceinline__ double ld(const void* v, int64_t e) {
    return __ldcs(static_cast<const double*>(v) + e);
  }
  static __device__ __forceinline__ double raw(const void* v, int64_t e) { return ld(v, e); }
};
template <>
struct XsVal<float> {  // FP32 values
  using AT = float;
  static __device__ __forceinline__ float ld(const void* v, int64_t e) {
    return __ldcs(static_cast<const float*>(v) + e);
  }
  static __device__ __forceinline__ float raw(const void* v, int64_t e) { return ld(v, e); }
};
template <>
struct XsVal<uint16_t> {  // BF16 values, FP32 arithmetic
  using AT = float;
  static __device__ __forceinline__ float ld(const void* v, int64_t e) {
    return __uint_as_float(static_cast<uint32_t>(__ldcs(static_cast<const unsigned short*>(v) + e)) << 16);
  }
  static __device__ __forceinline__ uint16_t raw(const void* v, int64_t e) {
    return __ldcs(static_cast<const unsigned short*>(v) + e);
  }
};

// A group of up to G consecutive steps of a cell, in registers; ns = the
// lane's steps in the group.  set(j, v) keeps step j's stored value, av(j)
// gives it in the arithmetic type.
template <typename ValT, int G>
struct XsGroup {
  using AT = typename XsVal<ValT>::AT;
  uint32_t id[G];
  AT a[G];
  int ns;
  __device__ __forceinline__ void set(int j, ValT v) { a[j] = static_cast<AT>(v); }
  __device__ __forceinline__ AT av(int j) const { return a[j]; }
};
// BF16: the raw 16-bit values, widened to FP32 only where the FMA uses them
// -- widening at load time would make the load phase wait for each load.
template <int G>
struct XsGroup<uint16_t, G> {
  using AT = float;
  uint32_t id[G];
  uint32_t a[G];
  int ns;
  __device__ __forceinline__ void set(int j, uint16_t v) { a[j] = v; }
  __device__ __forceinline__ float av(int j) const { return __uint_as_float(a[j] << 16); }
};

// Position of a group in a warp's stream over its (tile, half)'s slices: slice
// index i (into tl_slice), the cell (first entry st, S steps, fp = F | P << 6)
// and the first step s0 of the group; i = -1 past the end.  The cells of 32
// slices at a time sit in the lanes (lane l: slice index base + l), so finding
// the next slice with entries is a ballot.
struct XsPos {
  int i;
  int32_t st, S, fp, s0;
};

struct XsWindow {
  int base;  // slice index held by lane 0
  int32_t st, S, fp;
};

// A cell's layout word fp: with bit 31 set, full steps -- lanes 0..rem-1 hold
// S entries, the others S - 1 (rem = fp & 63), step s at first + 32 s; else
// dealt -- lanes 0..F-1 hold S entries, lane F holds P, the others none
// (F = fp & 63, P = fp >> 6), step s at first + s F + min(s, P).  In both,
// lane l's entry of step s is at first + s F + min(s, P) + l (F = 32, P = 0
// for full steps).
struct XsLayout {
  int32_t F, P, mine;  // mine: the lane's entries in the cell
};

__device__ __forceinline__ XsLayout xs_layout(int32_t S, int32_t fp, int lane) {
  XsLayout o;
  if (fp < 0) {
    const int32_t rem = fp & 63;
    o.F = 32;
    o.P = 0;
    o.mine = lane < rem ? S : S - 1;
  } else {
    o.F = fp & 63;
    o.P = fp >> 6;
    o.mine = lane < o.F ? S : (lane == o.F ? o.P : 0);
  }
  return o;
}

__device__ __forceinline__ void xs_window_load(const XsParams& p, int64_t g, int i_end, int base, int lane,
                                               XsWindow& w) {
  w.base = base;
  const int i = base + lane;
  if (i < i_end) {
    const int64_t key = g * p.nS + p.tl_slice[i];
    w.st = p.seg[key];
    w.S = p.seg[p.cells + key];
    w.fp = p.seg[2 * p.cells + key];
  } else {
    w.st = 0;
    w.S = 0;
    w.fp = 0;
  }
}

// The first group of the first slice index > i with entries of this warp.
__device__ __forceinline__ XsPos xs_next_slice(const XsParams& p, int64_t g, int i, int i_end, int lane,
                                               XsWindow& w) {
  while (true) {
    const int li = w.base + lane;
    const unsigned m = __ballot_sync(0xffffffffu, li > i && li < i_end && w.fp != 0);
    if (m) {
      const int src = __ffs(m) - 1;
      XsPos q;
      q.i = w.base + src;
      q.st = __shfl_sync(0xffffffffu, w.st, src);
      q.S = __shfl_sync(0xffffffffu, w.S, src);
      q.fp = __shfl_sync(0xffffffffu, w.fp, src);
      q.s0 = 0;
      return q;
    }
    if (w.base + 32 >= i_end) return XsPos{-1, 0, 0, 0, 0};
    xs_window_load(p, g, i_end, w.base + 32, lane, w);
  }
}

template <int G>
__device__ __forceinline__ XsPos xs_next(const XsParams& p, int64_t g, const XsPos& q, int i_end, int lane,
                                         XsWindow& w) {
  if (q.i < 0) return q;
  if (q.s0 + G < q.S) return XsPos{q.i, q.st, q.S, q.fp, q.s0 + G};
  return xs_next_slice(p, g, q.i, i_end, lane, w);
}

// Load the lane's entries of the group's steps (layout: xs_layout).  Full
// steps (nearly every cell) take one pointer per group and loads at constant
// offsets; dealt cells take the general position.
// FP32 values sit interleaved with their indices (one 8-byte entry); other
// value types in an array of their own.
template <typename ValT>
constexpr bool kXsIlv = sizeof(ValT) == 4;

// Bulk L2 prefetch of the n entries from a0 (multiples of 8: 16-byte bounds).
template <typename ValT>
__device__ __forceinline__ void xs_prefetch_entries(const XsParams& p, int64_t a0, int64_t n) {
  if constexpr (kXsIlv<ValT>) {
    prefetch_l2(p.idx + 2 * a0, static_cast<uint32_t>(n * 8));
  } else {
    prefetch_l2(p.idx + a0, static_cast<uint32_t>(n * 4));
    prefetch_l2(static_cast<const unsigned char*>(p.val) + a0 * static_cast<int64_t>(sizeof(ValT)),
                static_cast<uint32_t>(n * sizeof(ValT)));
  }
}

template <typename ValT>
__device__ __forceinline__ auto xs_val_ptr(const void* v) {
  if constexpr (sizeof(ValT) == 2)
    return static_cast<const unsigned short*>(v);
  else
    return static_cast<const ValT*>(v);
}

template <typename ValT, int G>
__device__ __forceinline__ void xs_load(const XsParams& p, const XsPos& q, int lane,
                                        XsGroup<ValT, G>& k) {
  if (q.fp < 0) {  // full steps: step s at first + 32 s
    const int32_t mine = lane < (q.fp & 63) ? q.S : q.S - 1;
    const int32_t ns = mine - q.s0;
    k.ns = ns < 0 ? 0 : (ns > G ? G : ns);
    const int64_t e0 = static_cast<int64_t>(q.st) + 32 * q.s0 + lane;
    if constexpr (kXsIlv<ValT>) {  // (index, value) in one 8-byte load
      const uint2* pe = reinterpret_cast<const uint2*>(p.idx) + e0;
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j < k.ns) {
          const uint2 w = __ldcs(pe + 32 * j);
          k.id[j] = w.x;
          k.set(j, __uint_as_float(w.y));
        }
      }
    } else {
      const uint32_t* pi = p.idx + e0;
      const auto* pv = xs_val_ptr<ValT>(p.val) + e0;
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j < k.ns) {
          k.id[j] = __ldcs(pi + 32 * j);
          k.set(j, static_cast<ValT>(__ldcs(pv + 32 * j)));
        }
      }
    }
    return;
  }
  const XsLayout lay = xs_layout(q.S, q.fp, lane);
  const int32_t F = lay.F, P = lay.P;
  const int32_t ns = lay.mine - q.s0;
  k.ns = ns < 0 ? 0 : (ns > G ? G : ns);
#pragma unroll
  for (int j = 0; j < G; ++j) {
    if (j < k.ns) {
      const int32_t s = q.s0 + j;
      const int64_t pos = static_cast<int64_t>(q.st) + static_cast<int64_t>(s) * F + (s < P ? s : P) + lane;
      if constexpr (kXsIlv<ValT>) {
        const uint2 w = __ldcs(reinterpret_cast<const uint2*>(p.idx) + pos);
        k.id[j] = w.x;
        k.set(j, __uint_as_float(w.y));
      } else {
        k.id[j] = __ldcs(p.idx + pos);
        k.set(j, XsVal<ValT>::raw(p.val, pos));
      }
    }
  }
}

// With large cells (the entries of a warp in a slice span several groups) a
// second cursor runs kXsAhead groups ahead of the loads and prefetches their
// entries into L2, so the loads find them there; with small cells its
// bookkeeping per group costs more than it hides.
constexpr int kXsAhead = 4;

template <typename ValT, int G>
__device__ __forceinline__ void xs_prefetch(const XsParams& p, const XsPos& q, int lane) {
  if (q.i < 0 || lane != 0) return;
  const XsLayout lay = xs_layout(q.S, q.fp, 0);
  const int32_t F = lay.F, P = lay.P;
  const int32_t s1 = q.s0 + G < q.S ? q.s0 + G : q.S;
  const int64_t e0 = static_cast<int64_t>(q.st) + static_cast<int64_t>(q.s0) * F + (q.s0 < P ? q.s0 : P);
  const int64_t e1 = static_cast<int64_t>(q.st) + static_cast<int64_t>(s1) * F + (s1 < P ? s1 : P);
  const int64_t a0 = e0 & ~int64_t(7), a1 = (e1 + 7) & ~int64_t(7);  // 16-byte bounds of both arrays
  xs_prefetch_entries<ValT>(p, a0, a1 - a0);
}

// Without the cursor: a warp's cells for consecutive slices lie back to back
// (cells are stored in (tile half, warp, slice) order), so its entries are one
// contiguous stream; each group prefetches into L2 a group's worth of that
// stream p.ahead entries past its own start, which can cover the DRAM latency
// of the loads a few groups later at the cost of two bulk prefetches.  The
// distance is the autotuner's pick per handle (0: off).

template <typename ValT, int G>
__device__ __forceinline__ void xs_ahead(const XsParams& p, const XsPos& q, int lane) {
  if (q.i < 0 || lane != 0 || p.ahead == 0) return;
  constexpr int64_t n = 32 * G;  // a multiple of 8 entries: 16-byte sizes in both arrays
  const int64_t a0 = (static_cast<int64_t>(q.st) + 32 * q.s0 + p.ahead) & ~int64_t(7);
  if (a0 + n > p.nent) return;
  xs_prefetch_entries<ValT>(p, a0, n);
}

// acc[a] += value * x[column] for the lane's steps of the group, then the
// warp synchronises (where two lanes' updates of one accumulator meet: the
// builder keeps them in different groups).  FP64: steps that continue the
// previous step's accumulator (kXsCont) add into a register, the accumulator
// is read at the first step of a run and written after its last (each FP64
// accumulator access costs two shared-memory wavefronts, so this pays there).
// FP32: the group's reads, sums and writes go in three passes, so the reads
// do not wait for the writes of earlier steps.
template <typename VT, typename ValT, int G>
__device__ __forceinline__ void xs_compute(const XsGroup<ValT, G>& k, const VT* __restrict__ xs, VT* acc) {
  VT xv[G];
#pragma unroll
  for (int j = 0; j < G; ++j)
    if (j < k.ns) xv[j] = xs[k.id[j] & kXsColMask];
  if constexpr (sizeof(VT) == 8) {
    VT sum = VT(0);
    VT* pa = acc;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (j < k.ns) {
        if (j == 0 || !(k.id[j] & kXsCont)) {  // a new accumulator (the first step of a group always is)
          if (j > 0) *pa = sum;
          pa = acc + (k.id[j] >> kXsColBits);
          sum = *pa;
        }
        sum = fma(static_cast<VT>(k.av(j)), xv[j], sum);
      }
    }
    if (k.ns > 0) *pa = sum;
  } else {
    // All of the group's accumulators are read first, then summed, then
    // written in step order: within a group a lane's steps on one accumulator
    // are consecutive (the builder keeps them so) and all but the first carry
    // kXsCont, so they add to the running value instead of the stale read.
    VT v[G];
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (j < k.ns) v[j] = acc[k.id[j] >> kXsColBits];
    VT run = VT(0);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (j < k.ns) {
        run = fma(static_cast<VT>(k.av(j)), xv[j], (j > 0 && (k.id[j] & kXsCont)) ? run : v[j]);
        v[j] = run;
      }
    }
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (j < k.ns) acc[k.id[j] >> kXsColBits] = v[j];
  }
  __syncwarp();
}

template <typename VT, typename ValT, int J, bool PF>
__global__ void __launch_bounds__(kXsThreads, 1) spmv_xslice_kernel(const XsParams p) {
  using AT = typename XsVal<ValT>::AT;
  constexpr int SC = XsCfg<VT, J>::kSliceCols;
  constexpr int NX = XsCfg<VT, J>::kBuffers;
  constexpr int G = XsCfg<VT, J>::kSteps;
  extern __shared__ __align__(128) unsigned char smem[];
  VT* xb = reinterpret_cast<VT*>(smem);  // [NX][SC]
  VT* acc = xb + NX * SC;                // accumulators of the tile's rows, then virtual rows
  const int q = blockIdx.x;              // (tile, half) = tile * J + half
  const int t = q / J;
  const int32_t tr0 = p.tile_row[t], R = p.tile_row[t + 1] - tr0;
  const int32_t nslots = p.vslot[q * (kXsWarps + 1) + kXsWarps];
  uint64_t* full = reinterpret_cast<uint64_t*>(acc + ((nslots + 31) & ~31));
  uint64_t* empty = full + NX;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < NX; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], kXsWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int i0 = p.tl_off[q], i1 = p.tl_off[q + 1];

  if (warp == kXsWarps) {  // ---------------------------------------- producer
    if (lane == 0) {
      const uint64_t pol = policy_evict_last();
      uint32_t v = 0;
      for (int i = i0; i < i1; ++i, ++v) {
        const int b = v % NX;
        if (v >= NX && !mbar_wait_bounded(&empty[b], (v / NX - 1) & 1u, p.status, p.wait_ns)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        const int64_t c0 = static_cast<int64_t>(p.tl_slice[i]) * SC;
        const int width = static_cast<int>(p.N - c0 < SC ? p.N - c0 : static_cast<int64_t>(SC));
        constexpr int kVec = 16 / sizeof(VT);
        const int wb = width / kVec * kVec;  // by bulk copy; the rest (< 16 bytes) by this thread
        VT* dst = xb + b * SC;
        const VT* src = static_cast<const VT*>(p.x) + c0;
        if (wb < width) {
          for (int k = wb; k < width; ++k) dst[k] = src[k];
          fence_proxy_async_smem();  // a later bulk copy may overwrite these addresses
        }
        mbar_arrive_expect_tx(&full[b], static_cast<uint32_t>(wb * sizeof(VT)));
        if (wb > 0) bulk_g2s(dst, src, static_cast<uint32_t>(wb * sizeof(VT)), &full[b], pol);
      }
      // copies still in flight land before the block can exit
      for (uint32_t u = v > NX ? v - NX : 0; u < v; ++u)
        mbar_wait_bounded(&full[u % NX], (u / NX) & 1u, p.status, p.wait_ns);
    }
    __syncwarp();
  } else {  // ------------------------------------------------------ consumers
    // Each warp keeps two groups in registers: while one is summed, the other
    // is in flight, across slice boundaries.  Slice i's buffer is waited for
    // before its first group is summed and released after its last; slices
    // without entries of this warp are waited for and released in turn, so
    // every warp arrives once per slice.
    const int64_t g = static_cast<int64_t>(q) * kXsWarps + warp;
    const int32_t r_lo = p.warp_row[q * (kXsWarps + 1) + warp] - tr0;
    const int32_t r_hi = p.warp_row[q * (kXsWarps + 1) + warp + 1] - tr0;
    const int32_t v_lo = p.vslot[q * (kXsWarps + 1) + warp], v_hi = p.vslot[q * (kXsWarps + 1) + warp + 1];
    for (int32_t r = r_lo + lane; r < r_hi; r += 32) acc[r] = VT(0);
    for (int32_t r = v_lo + lane; r < v_hi; r += 32) acc[r] = VT(0);
    __syncwarp();
    XsWindow win;
    xs_window_load(p, g, i1, i0, lane, win);
    // Two register groups with fixed roles, A and B, summed in turn: while one
    // is summed the other's loads are in flight.
    XsGroup<ValT, G> kA, kB;
    XsPos qA = xs_next_slice(p, g, i0 - 1, i1, lane, win);
    XsPos qB = xs_next<G>(p, g, qA, i1, lane, win);
    if (qA.i >= 0) xs_load<ValT, G>(p, qA, lane, kA);
    if (qB.i >= 0) xs_load<ValT, G>(p, qB, lane, kB);
    XsPos qn = xs_next<G>(p, g, qB, i1, lane, win);  // the group after the two in registers
    XsWindow winp;  // the prefetch cursor, kXsAhead groups ahead of the loads (PF)
    XsPos qp{-1, 0, 0, 0, 0};
    if constexpr (PF) {
      xs_window_load(p, g, i1, i0, lane, winp);
      qp = xs_next_slice(p, g, i0 - 1, i1, lane, winp);
      for (int d = 0; d < 2 + kXsAhead; ++d) {
        if (d >= 2) xs_prefetch<ValT, G>(p, qp, lane);
        qp = xs_next<G>(p, g, qp, i1, lane, winp);
      }
    }
    int i = i0;          // next slice to wait for
    int slot = 0;        // its ring slot
    uint32_t par = 0;    // and the phase parity of that slot's barrier
    int held = -1;       // slot of slice i - 1, waited for and not yet released (-1: none)
    bool ok = true;
    // Wait for slices up to `upto`, releasing the ones before.  A failed wait
    // (the launch's limit ran out) stops the warp's waits and, through the
    // flag, the producer's copies; the other warps' waits then run out too.
    auto advance_to = [&](int upto) {
      while (i <= upto) {
        if (held >= 0 && lane == 0 && ok) mbar_arrive(&empty[held]);
        if (ok && !__all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], par, p.status, p.wait_ns))) {
          ok = false;
          *abort_flag = 1;
        }
        held = slot;
        if (++slot == NX) {
          slot = 0;
          par ^= 1u;
        }
        ++i;
      }
    };
    while (qA.i >= 0) {
      advance_to(qA.i);
      if (ok) xs_compute<VT, ValT, G>(kA, xb + held * SC, acc);
      qA = qn;
      if (qA.i >= 0) xs_load<ValT, G>(p, qA, lane, kA);
      if constexpr (!PF) xs_ahead<ValT, G>(p, qA, lane);
      qn = xs_next<G>(p, g, qn, i1, lane, win);
      if constexpr (PF) {
        xs_prefetch<ValT, G>(p, qp, lane);
        qp = xs_next<G>(p, g, qp, i1, lane, winp);
      }
      if (qB.i < 0) break;
      advance_to(qB.i);
      if (ok) xs_compute<VT, ValT, G>(kB, xb + held * SC, acc);
      qB = qn;
      if (qB.i >= 0) xs_load<ValT, G>(p, qB, lane, kB);
      if constexpr (!PF) xs_ahead<ValT, G>(p, qB, lane);
      qn = xs_next<G>(p, g, qn, i1, lane, win);
      if constexpr (PF) {
        xs_prefetch<ValT, G>(p, qp, lane);
        qp = xs_next<G>(p, g, qp, i1, lane, winp);
      }
    }
    advance_to(i1 - 1);  // slices after this warp's last entries
    if (held >= 0 && lane == 0 && ok) mbar_arrive(&empty[held]);
    __syncwarp();
    // virtual rows back into their rows, each split row by one lane, in order
    if (ok) {
      const int32_t b1 = p.vl_off[g + 1];
      for (int32_t it = p.vl_off[g] + lane; it < b1; it += 32) {
        const int32_t rs = p.vl_item[3 * it], eb = p.vl_item[3 * it + 1], ec = p.vl_item[3 * it + 2];
        VT s = acc[rs];
        for (int32_t k = 0; k < ec; ++k) s += acc[eb + k];
        acc[rs] = s;
      }
    }
    __syncwarp();
    if constexpr (J == 1) {
      VT* y = static_cast<VT*>(p.y);
      if (ok)
        for (int32_t r = r_lo + lane; r < r_hi; r += 32) {
          const int32_t row = tr0 + r;
          y[p.yperm ? p.yperm[row] : row] = acc[r];
        }
    }
  }
  if constexpr (J == 2) {
    // Both halves of the tile are summed: each CTA writes half of the tile's
    // rows as the accumulator of CTA 0 plus that of CTA 1 (the same order in
    // both CTAs), one of them read from the partner's shared memory.
    cluster_sync_all();
    if (warp < kXsWarps && !*abort_flag) {
      const uint32_t me = cluster_rank();
      const uint32_t other = map_to_rank(acc, me ^ 1u);
      const int32_t half = (R + 1) / 2;
      const int32_t lo = static_cast<int32_t>(me) * half, hi = me ? R : (half < R ? half : R);
      VT* y = static_cast<VT*>(p.y);
      for (int32_t r = lo + static_cast<int32_t>(threadIdx.x); r < hi; r += 32 * kXsWarps) {
        const VT mine = acc[r];
        const VT theirs = ld_cluster(other + static_cast<uint32_t>(r * sizeof(VT)), VT(0));
        const int32_t row = tr0 + r;
        y[p.yperm ? p.yperm[row] : row] = me == 0 ? mine + theirs : theirs + mine;
      }
    }
    cluster_sync_all();  // the partner has read this CTA's accumulators
  }
}

// ------------------------------------------------------------- building

// cnt0[r] = entries of row r with column < split (columns ascending per row).
__global__ void xs_split_count_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      int32_t M, int32_t split, int32_t* __restrict__ cnt0) {
  const int32_t r = static_cast<int32_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= M) return;
  int32_t lo = rowptr[r], hi = rowptr[r + 1];
  const int32_t b = lo;
  while (lo < hi) {  // first entry with col >= split
    const int32_t mid = lo + (hi - lo) / 2;
    if (col[mid] < split)
      lo = mid + 1;
    else
      hi = mid;
  }
  cnt0[r] = lo - b;
}

// Per entry: its cell ((tile, half, warp), slice) and accumulator, and the sort
// key (cell << 15) | (accumulator % 32) << 10 | accumulator / 32: a cell's
// entries ordered by accumulator bank, then accumulator, then CSR (column) order.
__global__ void xs_key_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t M,
                              int64_t Z, const int32_t* __restrict__ tile_row, int32_t T, int J,
                              const int32_t* __restrict__ warp_row, const int32_t* __restrict__ cnt0,
                              const int32_t* __restrict__ rowinfo, int32_t split, int32_t SC, int32_t nS,
                              uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int32_t* __restrict__ counts) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= Z) return;
  int32_t lo = 0, hi = M;  // row: last r with rowptr[r] <= e
  while (hi - lo > 1) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (rowptr[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  const int32_t r = lo;
  int32_t tlo = 0, thi = T;  // tile: last t with tile_row[t] <= r
  while (thi - tlo > 1) {
    const int32_t mid = tlo + (thi - tlo) / 2;
    if (tile_row[mid] <= r)
      tlo = mid;
    else
      thi = mid;
  }
  const int32_t t = tlo;
  const int32_t c = col[e];
  const int h = (J == 2 && c >= split) ? 1 : 0;
  const int32_t qq = t * J + h;
  const int32_t* wr = warp_row + static_cast<int64_t>(qq) * (kXsWarps + 1);
  int32_t wlo = 0, whi = kXsWarps;  // warp: last w with wr[w] <= r (empty ranges skipped)
  while (whi - wlo > 1) {
    const int32_t mid = wlo + (whi - wlo) / 2;
    if (wr[mid] <= r)
      wlo = mid;
    else
      whi = mid;
  }
  const int32_t rank = static_cast<int32_t>(e - rowptr[r]) - (h ? (cnt0 ? cnt0[r] : 0) : 0);
  const int32_t info = rowinfo[static_cast<int64_t>(h) * M + r];
  const int32_t V = info & 127;
  int32_t slot = r - tile_row[t];
  if (V > 1) {
    const int32_t vv = rank % V;
    if (vv > 0) slot = (info >> 7) + vv - 1;
  }
  const int32_t s = c / SC;
  const int64_t cell = (static_cast<int64_t>(qq) * kXsWarps + wlo) * nS + s;
  keys[e] = (static_cast<uint64_t>(cell) << 15) | (static_cast<uint64_t>(slot & 31) << 10) |
            static_cast<uint64_t>(slot >> 5);
  vals[e] = static_cast<int32_t>(e);
  atomicAdd(counts + cell, 1);
}

// The longest run of equal keys (one accumulator's entries) in each cell.
__global__ void xs_mult_kernel(const uint64_t* __restrict__ keys, int64_t Z, int32_t* __restrict__ mult) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Z) return;
  const uint64_t k = keys[i];
  if (i > 0 && keys[i - 1] == k) return;
  int64_t j = i + 1;
  while (j < Z && keys[j] == k) ++j;
  atomicMax(mult + (k >> 15), static_cast<int32_t>(j - i));
}

// Lane and step of rank k of a cell when its runs cut the accumulator order
// (layout of xs_layout), and a lane's number of entries.
struct XsRun {
  int32_t lane, step;
};

__device__ __forceinline__ XsRun xs_run_of(int32_t k, int32_t S, int32_t fp) {
  XsRun r;
  if (fp < 0) {  // full steps: lanes 0..rem-1 hold S entries, the others S - 1 (S >= 2)
    const int32_t rem = fp & 63;
    if (k < rem * S) {
      r.lane = k / S;
      r.step = k - r.lane * S;
    } else {
      const int32_t k2 = k - rem * S;
      r.lane = rem + k2 / (S - 1);
      r.step = k2 - (r.lane - rem) * (S - 1);
    }
  } else {  // dealt: lane k / S, step k % S
    r.lane = k / S;
    r.step = k - r.lane * S;
  }
  return r;
}

__device__ __forceinline__ int32_t xs_lane_len(int32_t l, int32_t S, int32_t fp) {
  if (fp < 0) return l < (fp & 63) ? S : S - 1;
  const int32_t F = fp & 63;
  return l < F ? S : (l == F ? (fp >> 6) : 0);
}

// One thread per cell: the slot of every sorted entry (outpos).  A cell of at
// most 32 steps gets its accumulator groups (runs of equal keys) packed whole
// into the lane runs.  A lane's home is the accumulators of its shared-memory
// bank (the sort order groups them), so that the lanes of a step update
// different banks: the groups of two or more entries, largest first, go home
// when there is room, else into the run with the most room; then the single
// entries go home, and those whose home is full fill the room left.  If a
// group does not fit, the cell is tried again dealt over one or two more steps
// (more room per run).  Otherwise, and in longer cells, the runs cut the sort
// order where they end; a short cell that cannot be packed is first dealt over
// S >= m + G steps (m its largest accumulator count), so that a cut
// accumulator's two lanes meet at least a group boundary apart, as in the long
// cells.
constexpr int kXsPackBig = 128;  // groups of two or more entries a cell may have to be packed

__global__ void xs_pack_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ ustart,
                               const int32_t* __restrict__ counts, const int32_t* __restrict__ mult,
                               int32_t* __restrict__ seg, int64_t cells, int G, int32_t* __restrict__ outpos) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const int32_t n = counts[c];
  if (n == 0) return;
  const int32_t st = seg[c];
  int32_t S = seg[cells + c], fp = seg[2 * cells + c];
  const int64_t u0 = ustart[c];
  auto slot = [&](int32_t lane, int32_t step, int32_t F, int32_t P) {  // (F, P) of the layout
    return static_cast<int32_t>(st + step * F + (step < P ? step : P) + lane);
  };
  auto bank = [&](int64_t i) { return static_cast<int>((keys[i] >> 10) & 31u); };
  bool packed = false;
  if (S <= 32) {  // n <= 1024
    // the groups of two or more entries, largest first (insertion sort, stable)
    int32_t big_i[kXsPackBig], big_n[kXsPackBig];
    int nb = 0;
    bool fits_list = true;
    for (int64_t i = u0; i < u0 + n;) {
      int64_t j = i + 1;
      while (j < u0 + n && keys[j] == keys[i]) ++j;
      const int32_t m = static_cast<int32_t>(j - i);
      if (m > 1) {
        if (nb == kXsPackBig) {
          fits_list = false;
          break;
        }
        int q = nb++;
        while (q > 0 && big_n[q - 1] < m) {
          big_i[q] = big_i[q - 1];
          big_n[q] = big_n[q - 1];
          --q;
        }
        big_i[q] = static_cast<int32_t>(i - u0);
        big_n[q] = m;
      }
      i = j;
    }
    for (int extra = 0; fits_list && !packed && extra <= 2; ++extra) {
      int32_t S2 = S, fp2 = fp;
      if (extra > 0) {  // dealt over more steps
        S2 = S + extra;
        if (S2 > 32) break;
        const int32_t F2 = n / S2, P2 = n - F2 * S2;
        fp2 = F2 | (P2 << 6);
      }
      const int32_t F = fp2 < 0 ? 32 : (fp2 & 63), P = fp2 < 0 ? 0 : (fp2 >> 6);
      int32_t fill[32], room[32];
      for (int l = 0; l < 32; ++l) {
        fill[l] = 0;
        room[l] = xs_lane_len(l, S2, fp2);
      }
      auto place = [&](int64_t i0, int32_t m, int l) {
        for (int32_t t = 0; t < m; ++t) outpos[i0 + t] = slot(l, fill[l] + t, F, P);
        fill[l] += m;
        room[l] -= m;
      };
      bool ok = true;
      for (int b = 0; b < nb; ++b) {
        const int64_t i0 = u0 + big_i[b];
        int l = bank(i0);
        if (room[l] < big_n[b]) {
          l = 0;
          for (int q = 1; q < 32; ++q)
            if (room[q] > room[l]) l = q;
        }
        if (room[l] < big_n[b]) {
          ok = false;
          break;
        }
        place(i0, big_n[b], l);
      }
      if (!ok) continue;
      uint32_t deferred[32];  // single entries whose home was full (bit per entry of the cell)
      for (int w = 0; w < 32; ++w) deferred[w] = 0u;
      for (int64_t i = u0; i < u0 + n;) {
        int64_t j = i + 1;
        while (j < u0 + n && keys[j] == keys[i]) ++j;
        if (j - i == 1) {
          const int l = bank(i);
          if (room[l] > 0) {
            place(i, 1, l);
          } else {
            const int32_t r = static_cast<int32_t>(i - u0);
            deferred[r >> 5] |= 1u << (r & 31);
          }
        }
        i = j;
      }
      int l = 0;
      for (int w = 0; w < 32; ++w) {
        for (uint32_t bits = deferred[w]; bits; bits &= bits - 1) {
          while (l < 31 && room[l] == 0) ++l;  // the rooms add up to the deferred entries
          place(u0 + 32 * w + __ffs(bits) - 1, 1, l);
        }
      }
      packed = true;
      if (extra > 0) {
        seg[cells + c] = S2;
        seg[2 * cells + c] = fp2;
      }
    }
  }
  if (!packed) {
    if (S <= 32 && mult[c] > 1) {  // dealt over enough steps for cuts to meet a group boundary apart
      S = S > mult[c] + G ? S : mult[c] + G;
      const int32_t F2 = n / S, P2 = n - F2 * S;
      fp = F2 | (P2 << 6);
      seg[cells + c] = S;
      seg[2 * cells + c] = fp;
    }
    const int32_t F = fp < 0 ? 32 : (fp & 63), P = fp < 0 ? 0 : (fp >> 6);
    for (int32_t k = 0; k < n; ++k) {
      const XsRun r = xs_run_of(k, S, fp);
      outpos[u0 + k] = slot(r.lane, r.step, F, P);
    }
  }
}

// One warp per packed cell of full steps (at most 32): the order of each run's
// entries is free (an accumulator's entries are in one run), so it is chosen
// step by step to spread the shared-memory banks a step touches: at step s the
// lanes in turn take, among their remaining entries, the cheapest -- except
// that inside a register group of G steps a lane continues its previous
// accumulator while that has entries left, so that within a group each
// accumulator of a lane occupies consecutive steps (the kernel reads all of a
// group's accumulators before it writes any).  Without
// register runs (FP32 kernels) the cost is how often the entry's x bank plus
// its accumulator's bank are used at step s so far.  With register runs
// (FP64: cont = true) an entry that continues the lane's previous accumulator
// inside a register group touches no accumulator (cost: its x bank's uses);
// any other costs that plus two accesses of its accumulator's bank (one more
// for each earlier use).  Cells whose runs cut an accumulator keep their
// order.
constexpr int kXsOrderWarps = 8;  // warps (cells) per block

__global__ void __launch_bounds__(32 * kXsOrderWarps) xs_order_kernel(
    const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals, const int32_t* __restrict__ col,
    const int32_t* __restrict__ ustart, const int32_t* __restrict__ counts, const int32_t* __restrict__ seg,
    int64_t cells, int G, bool cont_runs, int32_t* __restrict__ outpos) {
  __shared__ int32_t use_x[kXsOrderWarps][32], use_a[kXsOrderWarps][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = static_cast<int64_t>(blockIdx.x) * kXsOrderWarps + w;
  if (c >= cells) return;  // the whole warp leaves together
  const int32_t n = counts[c], S = seg[cells + c], fp = seg[2 * cells + c];
  if (n == 0 || S > 32 || fp >= 0) return;  // full-step cells only
  const int32_t st = seg[c];
  const int64_t u0 = ustart[c];
  bool cut = false;  // packed cells only: no accumulator cut between two runs
  for (int64_t i = u0 + lane; i < u0 + n; i += 32) {
    const bool next_same = i + 1 < u0 + n && keys[i + 1] == keys[i];
    if (next_same && ((outpos[i] - st) & 31) != ((outpos[i + 1] - st) & 31)) cut = true;
  }
  if (__any_sync(0xffffffffu, cut)) return;
  // this lane's run: its entries' sorted positions and banks
  int32_t mine_i[32];
  uint16_t mine_k[32];  // the accumulator within the cell: bank << 10 | accumulator / 32
  uint8_t mine_x[32];
  int m = 0;
  for (int64_t i = u0; i < u0 + n; ++i) {
    if (((outpos[i] - st) & 31) != lane) continue;
    mine_i[m] = static_cast<int32_t>(i - u0);
    mine_x[m] = static_cast<uint8_t>(col[vals[i]] & 31);
    mine_k[m] = static_cast<uint16_t>(keys[i] & 0x7FFFu);
    ++m;
  }
  uint32_t taken = 0;
  int last = -1;  // the accumulator of the lane's previous pick
  __syncwarp();
  for (int s = 0; s < S; ++s) {
    use_x[w][lane] = 0;
    use_a[w][lane] = 0;
    __syncwarp();
    for (int turn = 0; turn < 32; ++turn) {
      if (lane == turn && s < m) {
        // inside a register group an accumulator's entries stay together: while
        // the lane's previous accumulator has entries left, one of them is next
        bool force = false;
        if (s % G != 0)
          for (int t = 0; t < m; ++t) force |= !((taken >> t) & 1u) && mine_k[t] == last;
        int best = -1, best_cost = 1 << 30;
        for (int t = 0; t < m; ++t) {
          if ((taken >> t) & 1u) continue;
          if (force && mine_k[t] != last) continue;
          const bool cont = cont_runs && s % G != 0 && mine_k[t] == last;
          const int cost = cont_runs ? use_x[w][mine_x[t]] + (cont ? 0 : 2 * (1 + use_a[w][mine_k[t] >> 10]))
                                     : use_x[w][mine_x[t]] + use_a[w][mine_k[t] >> 10];
          if (cost < best_cost) {
            best_cost = cost;
            best = t;
          }
        }
        taken |= 1u << best;
        ++use_x[w][mine_x[best]];
        if (!(cont_runs && s % G != 0 && mine_k[best] == last)) ++use_a[w][mine_k[best] >> 10];
        last = mine_k[best];
        outpos[u0 + mine_i[best]] = st + 32 * s + lane;
      }
      __syncwarp();
    }
  }
}

// One warp per cell: lane l marks the entries of its run that continue the
// accumulator of its previous step inside the same register group of G steps
// (kXsCont), so that the kernel keeps the running sum in a register there.
__global__ void xs_cont_kernel(const int32_t* __restrict__ seg, const int32_t* __restrict__ counts, int64_t cells,
                               int G, int stride, uint32_t* __restrict__ idx) {
  const int64_t c = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= cells || counts[c] == 0) return;
  const int32_t st = seg[c], S = seg[cells + c], fp = seg[2 * cells + c];
  const XsLayout lay = xs_layout(S, fp, lane);
  uint32_t prev = 0;
  for (int32_t s = 0; s < lay.mine; ++s) {
    const int64_t pos = static_cast<int64_t>(st) + static_cast<int64_t>(s) * lay.F + (s < lay.P ? s : lay.P) + lane;
    const uint32_t v = idx[pos * stride];
    if (s % G != 0 && (v >> kXsColBits) == (prev >> kXsColBits)) idx[pos * stride] = v | kXsCont;
    prev = v;
  }
}

// Sorted entry i goes to its slot: idx = (accumulator << 15) | column in slice;
// FP32 values interleaved with it (val_out null: entry pos is the 8 bytes
// idx_out[2 pos], idx_out[2 pos + 1]), other types in their own array.
__global__ void xs_scatter_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals, int64_t Z,
                                  const int32_t* __restrict__ outpos, const int32_t* __restrict__ col,
                                  const void* __restrict__ val, int vbytes, int32_t SC, int32_t nS,
                                  uint32_t* __restrict__ idx_out, void* __restrict__ val_out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Z) return;
  const uint64_t k = keys[i];
  const int64_t cell = static_cast<int64_t>(k >> 15);
  const int32_t slot = static_cast<int32_t>(((k & 1023u) << 5) | ((k >> 10) & 31u));
  const int32_t e = vals[i];
  const int64_t pos = outpos[i];
  const int32_t s = static_cast<int32_t>(cell % nS);
  const uint32_t id = (static_cast<uint32_t>(slot) << kXsColBits) | static_cast<uint32_t>(col[e] - s * SC);
  if (!val_out) {
    idx_out[2 * pos] = id;
    idx_out[2 * pos + 1] = __float_as_uint(static_cast<const float*>(val)[e]);
    return;
  }
  idx_out[pos] = id;
  if (vbytes == 8)
    static_cast<double*>(val_out)[pos] = static_cast<const double*>(val)[e];
  else if (vbytes == 4)
    static_cast<float*>(val_out)[pos] = static_cast<const float*>(val)[e];
  else
    static_cast<uint16_t*>(val_out)[pos] = static_cast<const uint16_t*>(val)[e];
}

int bit_width_u64(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Device arrays that are freed unless the build hands them to the handle.
struct OwnedSet {
  const Allocator& al;
  std::vector<void*> ptrs;
  explicit OwnedSet(const Allocator& a) : al(a) {}
  template <typename T>
  T* get(size_t count) {
    void* p = al.get(count * sizeof(T));
    if (p) ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void keep() { ptrs.clear(); }
  ~OwnedSet() {
    for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) al.put(*it);
  }
};

// Kernel attributes are set once per device and instantiation.
template <typename VT, typename ValT, int J>
maxe_status xs_prepare(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  if (device < 0 || device >= 64) return MAXE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (done[device]) return MAXE_OK;
  int optin = 0;
  MAXE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  MAXE_CUDA_TRY(cudaFuncSetAttribute(spmv_xslice_kernel<VT, ValT, J, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  MAXE_CUDA_TRY(cudaFuncSetAttribute(spmv_xslice_kernel<VT, ValT, J, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  done[device] = true;
  return MAXE_OK;
}

template <typename VT, typename ValT, int J>
maxe_status xs_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st) {
  MAXE_TRY((xs_prepare<VT, ValT, J>(h->device)));
  XsParams p{};
  p.idx = h->xs_idx;
  p.val = h->xs_val;
  p.seg = h->xs_seg;
  p.cells = h->xs_cells;
  p.nent = h->xs_nent;
  p.ahead = h->xs_ahead;
  p.tile_row = h->xs_tile_row;
  p.warp_row = h->xs_warp_row;
  p.vslot = h->xs_vslot;
  p.vl_off = h->xs_vl_off;
  p.vl_item = h->xs_vl_item;
  p.tl_off = h->xs_tl_off;
  p.tl_slice = h->xs_tl_slice;
  p.nS = h->xs_nS;
  p.N = h->cols;
  p.x = x;
  p.y = y;
  p.yperm = yperm;
  p.status = h->status;
  p.wait_ns = wait_limit_ns(h->device);
  const unsigned grid = static_cast<unsigned>(h->xs_ntiles) * J;
  const size_t smem = static_cast<size_t>(h->xs_smem);
  if constexpr (J == 1) {
    if (h->xs_prefetch)
      spmv_xslice_kernel<VT, ValT, 1, true><<<grid, kXsThreads, smem, st>>>(p);
    else
      spmv_xslice_kernel<VT, ValT, 1, false><<<grid, kXsThreads, smem, st>>>(p);
    MAXE_CUDA_TRY(cudaGetLastError());
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kXsThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (h->xs_prefetch)
      MAXE_CUDA_TRY(cudaLaunchKernelEx(&cfg, spmv_xslice_kernel<VT, ValT, 2, true>, p));
    else
      MAXE_CUDA_TRY(cudaLaunchKernelEx(&cfg, spmv_xslice_kernel<VT, ValT, 2, false>, p));
  }
  return MAXE_OK;
}

// Clusters of two CTAs of the pair kernel that the device runs at once.
template <typename ValT>
int pair_clusters(int device, int sms, size_t smem) {
  if (xs_prepare<float, ValT, 2>(device) != MAXE_OK) return sms / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * static_cast<unsigned>(sms));
  cfg.blockDim = dim3(kXsThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, spmv_xslice_kernel<float, ValT, 2, false>, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return sms / 2;
  }
  return n;
}

// Plan of one (tile, half): warp row ranges and virtual accumulators.
struct HalfPlan {
  int32_t warp_row[kXsWarps + 1];
  int32_t vslot[kXsWarps + 1];
  int64_t entries = 0;
};

// Warp ranges of rows [r0, r1) balanced on c[r] (entries in this half), and the
// virtual rows of each warp: a row with c > Tv = max(32, ceil(E_w / 96)) is
// split into V = ceil(c / Tv) <= 97 virtual rows; the first keeps the row's own
// accumulator (r - r0), the others take consecutive accumulators after the
// tile's rows.  With outputs: rowinfo[r] = V | first extra accumulator << 7 for
// split rows, and per warp its split rows (accumulator, first extra, V - 1)
// appended to items with the running count appended to vl_off.
void plan_half(const int32_t* c, int32_t r0, int32_t r1, std::vector<int64_t>& pre, HalfPlan& hp,
               int32_t* rowinfo, std::vector<int32_t>* items, std::vector<int32_t>* vl_off) {
  const int32_t R = r1 - r0;
  pre.resize(static_cast<size_t>(R) + 1);
  pre[0] = 0;
  for (int32_t r = 0; r < R; ++r) pre[r + 1] = pre[r] + c[r0 + r];
  const int64_t E = pre[R];
  hp.entries = E;
  int32_t prev = 0;
  for (int w = 0; w <= kXsWarps; ++w) {
    int32_t r = 0;
    if (w == kXsWarps) {
      r = R;
    } else if (w > 0) {
      const int64_t target = (E * w + kXsWarps - 1) / kXsWarps;
      r = static_cast<int32_t>(std::lower_bound(pre.begin(), pre.end(), target) - pre.begin());
      r = std::min(std::max(r, prev), R);
    }
    hp.warp_row[w] = r0 + r;
    prev = r;
  }
  int32_t next = R;
  for (int w = 0; w < kXsWarps; ++w) {
    hp.vslot[w] = next;
    const int32_t a = hp.warp_row[w] - r0, b = hp.warp_row[w + 1] - r0;
    const int64_t Ew = pre[b] - pre[a];
    const int64_t Tv = std::max<int64_t>(kXsVirtMin, (Ew + kXsVirtDiv - 1) / kXsVirtDiv);
    for (int32_t r = a; r < b; ++r) {
      const int64_t cr = c[r0 + r];
      if (cr <= Tv) continue;
      const int32_t V = static_cast<int32_t>((cr + Tv - 1) / Tv);
      if (rowinfo) rowinfo[r0 + r] = V | (next << 7);
      if (items) {
        items->push_back(r);
        items->push_back(next);
        items->push_back(V - 1);
      }
      next += V - 1;
    }
    if (vl_off) vl_off->push_back(static_cast<int32_t>(items->size() / 3));
  }
  hp.vslot[kXsWarps] = next;
}

// Build the x-sliced form with J column halves.  *built: 1 built, 0 not worth
// it (or not possible), -1 (J = 2 only) the halves of some tile are too uneven
// (unless force_pair).  force: build it even when its x traffic would be high.
template <typename VT, int J>
maxe_status build(maxe_handle* h, cudaStream_t st, bool force, bool force_pair, int* built) {
  constexpr int SC = XsCfg<VT, J>::kSliceCols;
  *built = 0;
  const int32_t M = h->rows, N = h->cols;
  const int64_t Z = h->nnz;
  if (M == 0 || N == 0 || Z == 0) return MAXE_OK;
  const int vb = value_bytes(h->dtype);
  const int32_t nS = static_cast<int32_t>(ceil_div(N, SC));
  const int32_t split = J == 2 ? (nS / 2) * SC : N;  // half 0: columns < split
  const Allocator& al = h->al;
  ScratchSet scratch(al);
  OwnedSet owned(al);
  // ---- accumulators a CTA can hold
  int optin = 0;
  MAXE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  const int64_t cap64 = (static_cast<int64_t>(optin) - static_cast<int64_t>(xs_ring_bytes<VT, J>()) - kXsBarBytes) /
                        static_cast<int64_t>(sizeof(VT));
  const int32_t cap = static_cast<int32_t>(std::min<int64_t>(cap64, kXsMaxSlots) & ~int64_t(31));
  if (cap < 64) return MAXE_OK;
  // ---- row pointers and (two halves) the entries of each row before the split, on the host
  std::vector<int32_t> rp(static_cast<size_t>(M) + 1), c0(static_cast<size_t>(M)), c1;
  MAXE_CUDA_TRY(cudaMemcpyAsync(rp.data(), h->rowptr, sizeof(int32_t) * (M + 1), cudaMemcpyDeviceToHost, st));
  int32_t* d_cnt0 = nullptr;
  if (J == 2) {
    d_cnt0 = scratch.get<int32_t>(M);
    if (!d_cnt0) return MAXE_ERR_OOM;
    xs_split_count_kernel<<<static_cast<unsigned>(ceil_div(M, 256)), 256, 0, st>>>(h->rowptr, h->col, M, split,
                                                                                  d_cnt0);
    MAXE_CUDA_TRY(cudaGetLastError());
    MAXE_CUDA_TRY(cudaMemcpyAsync(c0.data(), d_cnt0, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, st));
  }
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  if (J == 2) {
    c1.resize(static_cast<size_t>(M));
    for (int32_t r = 0; r < M; ++r) c1[r] = rp[r + 1] - rp[r] - c0[r];
  } else {
    for (int32_t r = 0; r < M; ++r) c0[r] = rp[r + 1] - rp[r];
  }
  // ---- tiles: nnz-balanced over the CTAs (pairs) the device runs at once,
  // cut shorter where the rows and virtual rows would not fit in shared memory
  int T_target = h->sms;
  if (J == 2)
    T_target = h->dtype == MAXE_BF16 ? pair_clusters<uint16_t>(h->device, h->sms, xs_smem_bytes<VT, J>(cap))
                                     : pair_clusters<float>(h->device, h->sms, xs_smem_bytes<VT, J>(cap));
  T_target = std::max(T_target, 1);
  std::vector<int32_t> trow{0};
  std::vector<HalfPlan> plans;
  std::vector<int64_t> pre;
  int32_t maxslots = 0;
  for (int32_t r0 = 0; r0 < M;) {
    const int32_t t = static_cast<int32_t>(trow.size()) - 1;
    const int64_t remaining_tiles = std::max<int64_t>(1, T_target - t);
    const int64_t target = rp[r0] + ceil_div(Z - rp[r0], remaining_tiles);
    int32_t r1 = static_cast<int32_t>(std::lower_bound(rp.begin() + r0 + 1, rp.end(), target) - rp.begin());
    r1 = std::max(std::min(r1, M), r0 + 1);
    r1 = static_cast<int32_t>(std::min<int64_t>(r1, static_cast<int64_t>(r0) + cap));
    HalfPlan hp[2];
    while (true) {
      int32_t need = 0;
      for (int hh = 0; hh < J; ++hh) {
        plan_half(hh == 0 ? c0.data() : c1.data(), r0, r1, pre, hp[hh], nullptr, nullptr, nullptr);
        need = std::max(need, hp[hh].vslot[kXsWarps]);
      }
      if (need <= cap || r1 == r0 + 1) {
        if (need > cap) return MAXE_OK;  // one row with more virtual rows than fit: leave the form unbuilt
        maxslots = std::max(maxslots, need);
        break;
      }
      r1 = std::max(r0 + 1, r1 - (need - cap) - 32);
    }
    for (int hh = 0; hh < J; ++hh) plans.push_back(hp[hh]);
    trow.push_back(r1);
    r0 = r1;
  }
  const int32_t T = static_cast<int32_t>(trow.size()) - 1;
  const int32_t Q = T * J;
  if (J == 2 && !force_pair) {  // both halves of every tile within 10% of their mean
    for (int32_t t = 0; t < T; ++t) {
      const int64_t a = plans[2 * t].entries, b = plans[2 * t + 1].entries;
      if (10 * std::max(a, b) > 11 * ((a + b) / 2) + 10) {
        *built = -1;
        return MAXE_OK;
      }
    }
  }
  // ---- virtual rows (per row and half), combine lists, warp ranges
  std::vector<int32_t> rowinfo(static_cast<size_t>(J) * M, 1), items, vl_off{0};
  std::vector<int32_t> wrow(static_cast<size_t>(Q) * (kXsWarps + 1)), vsl(static_cast<size_t>(Q) * (kXsWarps + 1));
  for (int32_t t = 0; t < T; ++t) {
    for (int hh = 0; hh < J; ++hh) {
      HalfPlan hp;
      plan_half(hh == 0 ? c0.data() : c1.data(), trow[t], trow[t + 1], pre, hp,
                rowinfo.data() + static_cast<size_t>(hh) * M, &items, &vl_off);
      const int32_t q = t * J + hh;
      for (int w = 0; w <= kXsWarps; ++w) {
        wrow[static_cast<size_t>(q) * (kXsWarps + 1) + w] = hp.warp_row[w];
        vsl[static_cast<size_t>(q) * (kXsWarps + 1) + w] = hp.vslot[w];
      }
    }
  }
  // ---- device copies of the plan
  const int64_t cells = static_cast<int64_t>(Q) * kXsWarps * nS;
  if (cells > (int64_t(1) << 40) || cells >= INT32_MAX) return MAXE_OK;
  int32_t* d_trow = owned.get<int32_t>(T + 1);
  int32_t* d_wv = owned.get<int32_t>(2 * wrow.size());  // warp rows, then virtual accumulators
  int32_t* d_vl = owned.get<int32_t>(vl_off.size() + std::max<size_t>(items.size(), 1));
  int32_t* d_info = scratch.get<int32_t>(rowinfo.size());
  if (!d_trow || !d_wv || !d_vl || !d_info) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_trow, trow.data(), sizeof(int32_t) * trow.size(), cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_wv, wrow.data(), sizeof(int32_t) * wrow.size(), cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_wv + wrow.size(), vsl.data(), sizeof(int32_t) * vsl.size(),
                                cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_vl, vl_off.data(), sizeof(int32_t) * vl_off.size(), cudaMemcpyHostToDevice, st));
  if (!items.empty())
    MAXE_CUDA_TRY(cudaMemcpyAsync(d_vl + vl_off.size(), items.data(), sizeof(int32_t) * items.size(),
                                  cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_info, rowinfo.data(), sizeof(int32_t) * rowinfo.size(), cudaMemcpyHostToDevice,
                                st));
  // ---- keys and counts
  uint64_t* keys = scratch.get<uint64_t>(Z);
  uint64_t* keys_alt = scratch.get<uint64_t>(Z);
  int32_t* vals = scratch.get<int32_t>(Z);
  int32_t* vals_alt = scratch.get<int32_t>(Z);
  int32_t* counts = scratch.get<int32_t>(2 * cells);  // counts, then longest accumulator run
  void* rs = scratch.get<unsigned char>(radix_scratch_bytes(Z));
  if (!keys || !keys_alt || !vals || !vals_alt || !counts || !rs) return MAXE_ERR_OOM;
  int32_t* mult = counts + cells;
  MAXE_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * cells, st));
  xs_key_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(
      h->rowptr, h->col, M, Z, d_trow, T, J, d_wv, d_cnt0, d_info, split, SC, nS, keys, vals, counts);
  MAXE_CUDA_TRY(cudaGetLastError());
  const int bits = 15 + bit_width_u64(static_cast<uint64_t>(cells - 1));
  MAXE_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, Z, bits, rs, st));
  xs_mult_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(keys, Z, mult);
  MAXE_CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> cnt(static_cast<size_t>(2 * cells));
  MAXE_CUDA_TRY(cudaMemcpyAsync(cnt.data(), counts, sizeof(int32_t) * 2 * cells, cudaMemcpyDeviceToHost, st));
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  // ---- cell descriptors (layout, aligned first entry), slices per (tile, half), the traffic estimate
  for (int64_t k = 0; k < cells; ++k) {
    if (cnt[k] >= (1 << 25)) return MAXE_OK;  // the layout word holds P < 2^25
  }
  constexpr int G = XsCfg<VT, J>::kSteps;
  std::vector<int32_t> seg(static_cast<size_t>(3 * cells)), ustart(static_cast<size_t>(cells));
  std::vector<int32_t> tl_off{0}, tl_slice;
  int64_t pos = 0, upos = 0, nonempty = 0;
  for (int64_t k = 0; k < cells; ++k) {
    const int32_t n = cnt[k], m = cnt[cells + k];
    int32_t S = 0, fp = 0;
    if (n > 0) {
      const int32_t L = static_cast<int32_t>(ceil_div(n, 32));
      if (L >= 2 && m <= L - 1 && (L <= 32 || m <= L - G)) {  // full steps
        S = L;
        fp = static_cast<int32_t>(0x80000000u | static_cast<uint32_t>(n - 32 * (L - 1)));
      } else {  // dealt: a run as long as the largest accumulator count
        S = std::max(L, m);
        if (S > 32) S = std::max(S, m + G);
        const int32_t F = n / S, P = n - F * S;
        fp = F | (P << 6);
      }
    }
    seg[k] = static_cast<int32_t>(pos);
    seg[cells + k] = S;
    seg[2 * cells + k] = fp;
    ustart[k] = static_cast<int32_t>(upos);
    pos = round_up(pos + n, 8);  // every cell starts on a 32-byte sector of the index array
    upos += n;
    nonempty += n > 0;
  }
  const int64_t Zp = pos;
  for (int32_t q = 0; q < Q; ++q) {
    for (int32_t s = 0; s < nS; ++s) {
      int64_t any = 0;
      for (int w = 0; w < kXsWarps; ++w) any += cnt[(static_cast<int64_t>(q) * kXsWarps + w) * nS + s];
      if (any) tl_slice.push_back(s);
    }
    tl_off.push_back(static_cast<int32_t>(tl_slice.size()));
  }
  const int64_t matrix_bytes = Z * (vb + 4);
  const int64_t x_bytes = static_cast<int64_t>(tl_slice.size()) * sizeof(VT) * SC;
  if (!force && x_bytes > 8 * matrix_bytes) return MAXE_OK;  // the CSR kernel will do better
  if (Zp + kXsSlack > INT32_MAX) return MAXE_OK;
  // ---- the format's arrays (FP32 values: one array of 8-byte (index, value) entries)
  const bool ilv = h->dtype == MAXE_F32;
  uint32_t* idx = owned.get<uint32_t>((ilv ? 2 : 1) * (Zp + kXsSlack));
  void* xval = ilv ? nullptr : owned.get<unsigned char>(static_cast<size_t>(vb) * (Zp + kXsSlack));
  int32_t* d_seg = owned.get<int32_t>(3 * cells);
  int32_t* d_tl = owned.get<int32_t>(tl_off.size() + std::max<size_t>(tl_slice.size(), 1));
  int32_t* d_ustart = scratch.get<int32_t>(cells);
  int32_t* outpos = vals_alt;  // the sort's ping-pong values are free after it
  if (!idx || (!ilv && !xval) || !d_seg || !d_tl || !d_ustart) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_seg, seg.data(), sizeof(int32_t) * 3 * cells, cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_ustart, ustart.data(), sizeof(int32_t) * cells, cudaMemcpyHostToDevice, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(d_tl, tl_off.data(), sizeof(int32_t) * tl_off.size(), cudaMemcpyHostToDevice, st));
  if (!tl_slice.empty())
    MAXE_CUDA_TRY(cudaMemcpyAsync(d_tl + tl_off.size(), tl_slice.data(), sizeof(int32_t) * tl_slice.size(),
                                  cudaMemcpyHostToDevice, st));
  // gaps between cells and the slack after the last one hold zeros
  MAXE_CUDA_TRY(cudaMemsetAsync(idx, 0, sizeof(uint32_t) * (ilv ? 2 : 1) * (Zp + kXsSlack), st));
  if (!ilv) MAXE_CUDA_TRY(cudaMemsetAsync(xval, 0, static_cast<size_t>(vb) * (Zp + kXsSlack), st));
  xs_pack_kernel<<<static_cast<unsigned>(ceil_div(cells, 128)), 128, 0, st>>>(keys, d_ustart, counts, mult, d_seg,
                                                                              cells, G, outpos);
  MAXE_CUDA_TRY(cudaGetLastError());
  xs_order_kernel<<<static_cast<unsigned>(ceil_div(cells, kXsOrderWarps)), 32 * kXsOrderWarps, 0, st>>>(
      keys, vals, h->col, d_ustart, counts, d_seg, cells, G, sizeof(VT) == 8, outpos);
  MAXE_CUDA_TRY(cudaGetLastError());
  xs_scatter_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(keys, vals, Z, outpos, h->col, h->val,
                                                                             vb, SC, nS, idx, xval);
  MAXE_CUDA_TRY(cudaGetLastError());
  xs_cont_kernel<<<static_cast<unsigned>(ceil_div(cells * 32, 256)), 256, 0, st>>>(d_seg, counts, cells, G,
                                                                                   ilv ? 2 : 1, idx);
  MAXE_CUDA_TRY(cudaGetLastError());
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors and scratch go out of scope
  owned.keep();
  h->xs_idx = idx;
  h->xs_val = xval;
  h->xs_seg = d_seg;
  h->xs_cells = cells;
  h->xs_tile_row = d_trow;
  h->xs_warp_row = d_wv;
  h->xs_vslot = d_wv + wrow.size();
  h->xs_vl_off = d_vl;
  h->xs_vl_item = d_vl + vl_off.size();
  h->xs_tl_off = d_tl;
  h->xs_tl_slice = d_tl + tl_off.size();
  h->xs_ntiles = T;
  h->xs_nS = nS;
  h->xs_pair = J;
  h->xs_smem = static_cast<int32_t>(xs_smem_bytes<VT, J>((maxslots + 31) & ~31));
  h->xs_bytes = Zp * (4 + vb) + 12 * cells;
  h->xs_nent = Zp + kXsSlack;
  constexpr int64_t kPrefetchCell = 2 * 32 * XsCfg<VT, J>::kSteps;  // mean entries per cell from which the cursor runs
  h->xs_prefetch = nonempty > 0 && Z >= kPrefetchCell * nonempty ? 1 : 0;
  *built = 1;
  return MAXE_OK;
}

}  // namespace

maxe_status xslice_build(maxe_handle* h, cudaStream_t st, bool force, int pairs) {
  int built = 0;
  maxe_status s = MAXE_OK;
  if (h->dtype == MAXE_F64) {
    s = build<double, 1>(h, st, force, false, &built);
  } else {
    if (pairs >= 0) s = build<float, 2>(h, st, force, pairs > 0, &built);
    if (s == MAXE_OK && built <= 0 && pairs <= 0) s = build<float, 1>(h, st, force, false, &built);
  }
  if (s == MAXE_OK && built > 0) h->xs_use = 1;
  return s;
}

bool xslice_ready(const maxe_handle* h, const void* x) {
  return h->xs_idx && h->xs_use && (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
}

maxe_status xslice_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st) {
  if (h->dtype == MAXE_F64) return xs_launch<double, double, 1>(h, x, y, yperm, st);
  if (h->xs_pair == 2) {
    if (h->dtype == MAXE_F32) return xs_launch<float, float, 2>(h, x, y, yperm, st);
    return xs_launch<float, uint16_t, 2>(h, x, y, yperm, st);
  }
  if (h->dtype == MAXE_F32) return xs_launch<float, float, 1>(h, x, y, yperm, st);
  return xs_launch<float, uint16_t, 1>(h, x, y, yperm, st);
}

void xslice_release(maxe_handle* h) {
  const Allocator& al = h->al;
  al.put(h->xs_tl_off);
  al.put(h->xs_seg);
  al.put(h->xs_val);
  al.put(h->xs_idx);
  al.put(h->xs_vl_off);
  al.put(h->xs_warp_row);
  al.put(h->xs_tile_row);
  h->xs_tl_off = h->xs_tl_slice = h->xs_seg = nullptr;
  h->xs_vl_off = h->xs_vl_item = nullptr;
  h->xs_warp_row = h->xs_vslot = h->xs_tile_row = nullptr;
  h->xs_idx = nullptr;
  h->xs_val = nullptr;
  h->xs_use = 0;
  h->xs_pair = 1;
}

}  // namespace maxe
