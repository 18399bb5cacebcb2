// spmv.cu -- nnz-balanced CSR SpMV / SpMM on the permuted matrix (Section 2:
// y_i = sum_{l in ROW[i]:ROW[i+1]} V[l] * x[COL[l]];  Eq. 1 for the permuted form).
//
// Work partition.  The nonzeros are cut into fixed chunks of kChunk = 2048
// entries.  Chunk q owns the rows whose last entry falls inside it (rows with
// rowptr[r+1] in (q*C, (q+1)*C]; chunk 0 also owns leading empty rows), so
// every row is written by exactly one chunk:  chunk_row[q] = first row with
// rowptr[r+1] > q*C.  A launch of G persistent CTAs gives CTA c the chunk range
// [c*nq/G, (c+1)*nq/G): equal nonzeros per CTA whatever the row lengths, which
// is the load balance the paper's laggard argument asks of the permutation
// (Section 1), obtained here without it.
//
// Pipeline per CTA (288 threads): one producer warp streams each chunk's COL and
// VAL slices and its slice of ROW into shared memory with 1-D bulk copies (TMA),
// S stages deep, completion on mbarriers, L2 evict-first (the matrix is read once
// per product).  Eight consumer warps, each thread holding 8 consecutive entries:
//   1. mark the first entry of every row that starts in the chunk (bit flags);
//   2. gather x[COL] (through L1/L2) and form the products in registers;
//   3. segmented inclusive scan of the products: serial over the thread's 8
//      entries, warp shuffles across lanes, one shared-memory step across warps;
//      the partial row that crosses from the previous chunk enters as a carry;
//   4. y[row] = scan value at the row's last entry, for every owned row
//      (empty rows get 0; rows may be scattered through rperm, which fuses the
//      y = P_r^{-1} y' step of Eq. 1 into the epilogue).
// A row that starts before the CTA's first chunk is summed directly from HBM by
// the CTA before its pipeline starts, so CTAs never exchange partial sums and
// the result depends only on the matrix, the chunk size and G: it is
// deterministic.
//
// SpMM reuses the pipeline: X rows are gathered VW columns at a time (float4,
// float2/double2), and the scan runs on VW-wide vectors, one pass per group of
// VW columns.
#include <algorithm>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;  // 256
constexpr int kThreads = kConsumers + 32;        // + producer warp
constexpr int kItems = 8;                        // entries per consumer thread
constexpr int kRowCap = kChunk / 2 + 8;          // rowptr slice held in shared memory
constexpr int kMaxK = 64;                        // right-hand sides per call
constexpr int kBarConsumers = 1;                 // named barrier id
static_assert(kConsumers * kItems == kChunk, "chunk = consumers x items");

template <typename VT>
struct Acc;
template <>
struct Acc<double> {
  using T = double;
};
template <>
struct Acc<float> {
  using T = float;
};
template <>
struct Acc<uint16_t> {
  using T = float;
};

struct Params {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  const void* X;
  void* Y;
  const int32_t* yperm;
  const int32_t* chunk_row;
  unsigned* status;
  int64_t ldx, ldy, Z;
  int32_t k, M, nq;
};

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename VT, int VW, int S>
struct Layout {
  using AT = typename Acc<VT>::T;
  static constexpr size_t col_off = 0;
  static constexpr size_t val_off = col_off + size_t(S) * kChunk * 4;
  static constexpr size_t rp_off = align16(val_off + size_t(S) * kChunk * sizeof(VT));
  static constexpr size_t sums_off = align16(rp_off + size_t(S) * kRowCap * 4);
  static constexpr size_t flags_off = align16(sums_off + size_t(kChunk) * VW * sizeof(AT));
  static constexpr size_t wagg_off = align16(flags_off + (kChunk / 32) * 4);
  static constexpr size_t waggf_off = align16(wagg_off + kConsumerWarps * VW * sizeof(AT));
  static constexpr size_t carry_off = align16(waggf_off + kConsumerWarps * 4);
  static constexpr size_t meta_off = align16(carry_off + (kMaxK + 4) * sizeof(AT));
  static constexpr size_t bar_off = align16(meta_off + S * sizeof(int4));
  static constexpr size_t bytes = bar_off + 2 * S * sizeof(uint64_t);
};

// ---- value / vector access ------------------------------------------------
template <typename VT, typename AT>
__device__ __forceinline__ AT to_acc(VT v) {
  return static_cast<AT>(v);
}
template <>
__device__ __forceinline__ float to_acc<uint16_t, float>(uint16_t v) {
  return bf16_bits_to_float(v);
}

// 8 consecutive values from shared memory (16-byte aligned).
template <typename VT, typename AT>
__device__ __forceinline__ void load8(const VT* p, AT (&a)[kItems]);
template <>
__device__ __forceinline__ void load8<float, float>(const float* p, float (&a)[kItems]) {
  const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
  a[0] = u.x, a[1] = u.y, a[2] = u.z, a[3] = u.w, a[4] = v.x, a[5] = v.y, a[6] = v.z, a[7] = v.w;
}
template <>
__device__ __forceinline__ void load8<double, double>(const double* p, double (&a)[kItems]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 u = reinterpret_cast<const double2*>(p)[i];
    a[2 * i] = u.x, a[2 * i + 1] = u.y;
  }
}
template <>
__device__ __forceinline__ void load8<uint16_t, float>(const uint16_t* p, float (&a)[kItems]) {
  const uint4 u = reinterpret_cast<const uint4*>(p)[0];
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[2 * i] = __uint_as_float(w[i] << 16);
    a[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

template <int VW, typename AT>
__device__ __forceinline__ void xload(const AT* __restrict__ X, int32_t c, int64_t ldx, int c0, int k, AT (&xv)[VW]) {
  const AT* px = X + static_cast<int64_t>(c) * ldx + c0;
  if constexpr (VW == 1) {
    xv[0] = __ldg(px);
  } else {
    if (c0 + VW <= k) {
      if constexpr (VW == 2 && sizeof(AT) == 4) {
        const float2 u = __ldg(reinterpret_cast<const float2*>(px));
        xv[0] = u.x, xv[1] = u.y;
      } else if constexpr (VW == 2 && sizeof(AT) == 8) {
        const double2 u = __ldg(reinterpret_cast<const double2*>(px));
        xv[0] = u.x, xv[1] = u.y;
      } else {
        const float4 u = __ldg(reinterpret_cast<const float4*>(px));
        xv[0] = u.x, xv[1] = u.y, xv[2] = u.z, xv[3] = u.w;
      }
    } else {
#pragma unroll
      for (int w = 0; w < VW; ++w) xv[w] = (c0 + w < k) ? __ldg(px + w) : AT(0);
    }
  }
}

template <int VW, typename AT>
__device__ __forceinline__ void ystore(AT* __restrict__ Y, int64_t row, int64_t ldy, int c0, int k,
                                       const AT (&v)[VW]) {
  AT* py = Y + row * ldy + c0;
  if constexpr (VW == 1) {
    *py = v[0];
  } else {
    if (c0 + VW <= k) {
      if constexpr (VW == 2 && sizeof(AT) == 4) {
        *reinterpret_cast<float2*>(py) = make_float2(v[0], v[1]);
      } else if constexpr (VW == 2 && sizeof(AT) == 8) {
        *reinterpret_cast<double2*>(py) = make_double2(v[0], v[1]);
      } else {
        *reinterpret_cast<float4*>(py) = make_float4(v[0], v[1], v[2], v[3]);
      }
    } else {
#pragma unroll
      for (int w = 0; w < VW; ++w)
        if (c0 + w < k) py[w] = v[w];
    }
  }
}

// ---- producer warp --------------------------------------------------------
template <typename VT, int VW, int S>
__device__ __forceinline__ void produce(const Params& p, unsigned char* sm, int64_t q0, int64_t q1) {
  using L = Layout<VT, VW, S>;
  const int lane = threadIdx.x & 31;
  int32_t* col_s = reinterpret_cast<int32_t*>(sm + L::col_off);
  VT* val_s = reinterpret_cast<VT*>(sm + L::val_off);
  int32_t* rp_s = reinterpret_cast<int32_t*>(sm + L::rp_off);
  int4* meta = reinterpret_cast<int4*>(sm + L::meta_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L::bar_off);
  uint64_t* empty = full + S;
  const VT* val_g = static_cast<const VT*>(p.val);
  const uint64_t pol = policy_evict_first();
  const int64_t n = q1 - q0;
  int abort = 0;
  for (int64_t base = 0; base < n && !abort; base += 32) {
    const int64_t qa = q0 + base + lane;
    const int32_t cra = (qa <= q1) ? p.chunk_row[qa] : 0;
    const int32_t crb = (qa + 1 <= q1) ? p.chunk_row[qa + 1] : 0;
    const int cnt = static_cast<int>(n - base < 32 ? n - base : 32);
    for (int j = 0; j < cnt; ++j) {
      const int32_t ra = __shfl_sync(0xffffffffu, cra, j);
      const int32_t rb = __shfl_sync(0xffffffffu, crb, j);
      if (lane == 0) {
        const int64_t i = base + j;
        const int s = static_cast<int>(i % S);
        if (i >= S && !mbar_wait_bounded(&empty[s], static_cast<uint32_t>(((i / S) & 1) ^ 1), p.status)) abort = 1;
        if (!abort) {
          const int64_t q = q0 + i;
          const int32_t lo = ra & ~3;
          const int32_t hi = (rb + 4) & ~3;
          const int32_t nr = hi - lo;
          const int big = nr > kRowCap;
          meta[s] = make_int4(ra, rb, lo, big);
          const uint32_t bytes = kChunk * 4u + kChunk * static_cast<uint32_t>(sizeof(VT)) + (big ? 0u : nr * 4u);
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_g2s(col_s + static_cast<size_t>(s) * kChunk, p.col + q * kChunk, kChunk * 4u, &full[s], pol);
          bulk_g2s(val_s + static_cast<size_t>(s) * kChunk, val_g + q * kChunk,
                   kChunk * static_cast<uint32_t>(sizeof(VT)), &full[s], pol);
          if (!big) bulk_g2s(rp_s + static_cast<size_t>(s) * kRowCap, p.rowptr + lo, nr * 4u, &full[s], pol);
        }
      }
      abort = __shfl_sync(0xffffffffu, abort, 0);
      if (abort) break;
    }
  }
}

// ---- consumer warps -------------------------------------------------------
template <typename VT, int VW, int S>
__device__ __forceinline__ void consume(const Params& p, unsigned char* sm, int64_t q0, int64_t q1) {
  using L = Layout<VT, VW, S>;
  using AT = typename Acc<VT>::T;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int32_t* col_s = reinterpret_cast<const int32_t*>(sm + L::col_off);
  const VT* val_s = reinterpret_cast<const VT*>(sm + L::val_off);
  const int32_t* rp_s = reinterpret_cast<const int32_t*>(sm + L::rp_off);
  AT* sums = reinterpret_cast<AT*>(sm + L::sums_off);
  uint32_t* flags = reinterpret_cast<uint32_t*>(sm + L::flags_off);
  AT* wagg = reinterpret_cast<AT*>(sm + L::wagg_off);
  int* waggf = reinterpret_cast<int*>(sm + L::waggf_off);
  AT* carry = reinterpret_cast<AT*>(sm + L::carry_off);
  const int4* meta = reinterpret_cast<const int4*>(sm + L::meta_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L::bar_off);
  uint64_t* empty = full + S;

  const AT* X = static_cast<const AT*>(p.X);
  AT* Y = static_cast<AT*>(p.Y);
  const VT* val_g = static_cast<const VT*>(p.val);
  const int k = p.k;
  const int ngroups = (k + VW - 1) / VW;

  // Carry into the first chunk: the part of its first row lying before it.
  {
    const int64_t qc0 = q0 * kChunk;
    const int32_t r = p.chunk_row[q0];
    const int64_t st = (r < p.M) ? static_cast<int64_t>(p.rowptr[r]) : qc0;
    for (int g = 0; g < ngroups; ++g) {
      AT acc[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) acc[u] = AT(0);
      for (int64_t e = st + tid; e < qc0; e += kConsumers) {
        AT xv[VW];
        xload<VW>(X, p.col[e], p.ldx, g * VW, k, xv);
        const AT a = to_acc<VT, AT>(val_g[e]);
#pragma unroll
        for (int u = 0; u < VW; ++u) acc[u] += a * xv[u];
      }
#pragma unroll
      for (int u = 0; u < VW; ++u)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], d);
      if (lane == 0)
#pragma unroll
        for (int u = 0; u < VW; ++u) wagg[w * VW + u] = acc[u];
      named_bar(kBarConsumers, kConsumers);
      if (tid < VW) {
        AT t = AT(0);
        for (int ww = 0; ww < kConsumerWarps; ++ww) t += wagg[ww * VW + tid];
        carry[g * VW + tid] = t;
      }
      named_bar(kBarConsumers, kConsumers);
    }
    if (tid < kChunk / 32) flags[tid] = 0u;
    named_bar(kBarConsumers, kConsumers);
  }

  const int64_t n = q1 - q0;
  for (int64_t i = 0; i < n; ++i) {
    const int s = static_cast<int>(i % S);
    bool ok = mbar_wait_bounded(&full[s], static_cast<uint32_t>((i / S) & 1), p.status);
    ok = named_bar_and(kBarConsumers, kConsumers, ok);
    if (!ok) return;
    const int4 m = meta[s];
    const int32_t ra = m.x, rb = m.y;
    const int32_t* rp = m.w ? p.rowptr : (rp_s + static_cast<size_t>(s) * kRowCap - m.z);
    const int64_t qC = (q0 + i) * kChunk;

    // 1. row-start flags of the chunk
    for (int32_t r = ra + tid; r <= rb && r < p.M; r += kConsumers) {
      const int64_t st = rp[r];
      if (st >= qC && st < qC + kChunk) {
        const bool nonempty = (r < rb) ? (rp[r + 1] > st) : true;
        if (nonempty) {
          const int off = static_cast<int>(st - qC);
          atomicOr(&flags[off >> 5], 1u << (off & 31));
        }
      }
    }
    named_bar(kBarConsumers, kConsumers);
    const uint32_t f8 = (flags[tid >> 2] >> ((tid & 3) * 8)) & 0xFFu;

    int32_t cj[kItems];
    AT a[kItems];
    {
      const int4* cp = reinterpret_cast<const int4*>(col_s + static_cast<size_t>(s) * kChunk + kItems * tid);
      const int4 c0v = cp[0], c1v = cp[1];
      cj[0] = c0v.x, cj[1] = c0v.y, cj[2] = c0v.z, cj[3] = c0v.w;
      cj[4] = c1v.x, cj[5] = c1v.y, cj[6] = c1v.z, cj[7] = c1v.w;
      load8<VT, AT>(val_s + static_cast<size_t>(s) * kChunk + kItems * tid, a);
    }
    const int64_t e0 = qC + kItems * tid;
    const int nvalid = static_cast<int>(p.Z - e0 < 0 ? 0 : (p.Z - e0 > kItems ? kItems : p.Z - e0));

    for (int g = 0; g < ngroups; ++g) {
      const int c0 = g * VW;
      // 2. products
      AT v[kItems][VW];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        if (j < nvalid) {
          AT xv[VW];
          xload<VW>(X, cj[j], p.ldx, c0, k, xv);
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] = a[j] * xv[u];
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] = AT(0);
        }
      }
      // 3a. serial segmented scan over the thread's entries
#pragma unroll
      for (int j = 1; j < kItems; ++j)
        if (!((f8 >> j) & 1u))
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] += v[j - 1][u];
      // 3b. warp-level segmented scan of the thread aggregates
      int F = f8 != 0u;
      AT V[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) V[u] = v[kItems - 1][u];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int Fu = __shfl_up_sync(0xffffffffu, F, d);
        AT Vu[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) Vu[u] = __shfl_up_sync(0xffffffffu, V[u], d);
        if (lane >= d) {
          if (!F)
#pragma unroll
            for (int u = 0; u < VW; ++u) V[u] += Vu[u];
          F |= Fu;
        }
      }
      int Fe = __shfl_up_sync(0xffffffffu, F, 1);
      AT Ve[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) Ve[u] = __shfl_up_sync(0xffffffffu, V[u], 1);
      if (lane == 0) {
        Fe = 0;
#pragma unroll
        for (int u = 0; u < VW; ++u) Ve[u] = AT(0);
      }
      if (lane == 31) {
        waggf[w] = F;
#pragma unroll
        for (int u = 0; u < VW; ++u) wagg[w * VW + u] = V[u];
      }
      named_bar(kBarConsumers, kConsumers);
      if (g == 0 && tid < kChunk / 32) flags[tid] = 0u;  // every thread has its f8 by now
      // 3c. prefix = carry (+) warps before w (+) lanes before this one
      AT P[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) P[u] = carry[c0 + u];
      for (int ww = 0; ww < w; ++ww) {
        const bool fw = waggf[ww] != 0;
#pragma unroll
        for (int u = 0; u < VW; ++u) P[u] = fw ? wagg[ww * VW + u] : P[u] + wagg[ww * VW + u];
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) P[u] = Fe ? Ve[u] : P[u] + Ve[u];
      const int first_flag = f8 ? __ffs(f8) - 1 : kItems;
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (j < first_flag)
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] += P[u];
      AT* sp = sums + static_cast<size_t>(kItems * tid) * VW;
#pragma unroll
      for (int j = 0; j < kItems; ++j)
#pragma unroll
        for (int u = 0; u < VW; ++u) sp[j * VW + u] = v[j][u];
      named_bar(kBarConsumers, kConsumers);
      // 4. owned rows
      for (int32_t r = ra + tid; r < rb; r += kConsumers) {
        const int32_t st = rp[r], en = rp[r + 1];
        AT out[VW];
        if (en > st) {
          const AT* src = sums + static_cast<size_t>(en - 1 - qC) * VW;
#pragma unroll
          for (int u = 0; u < VW; ++u) out[u] = src[u];
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) out[u] = AT(0);
        }
        const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[r]) : static_cast<int64_t>(r);
        ystore<VW>(Y, row, p.ldy, c0, k, out);
      }
      if (tid == 0) {
        const bool cont = (rb < p.M) && (rp[rb] < qC + kChunk);
#pragma unroll
        for (int u = 0; u < VW; ++u) carry[c0 + u] = cont ? sums[static_cast<size_t>(kChunk - 1) * VW + u] : AT(0);
      }
      named_bar(kBarConsumers, kConsumers);
    }
    if (tid == 0) mbar_arrive(&empty[s]);
  }
}

template <typename VT, int VW, int S>
__global__ void __launch_bounds__(kThreads) spmm_chunk_kernel(Params p) {
  extern __shared__ __align__(128) unsigned char sm[];
  using L = Layout<VT, VW, S>;
  const int64_t G = gridDim.x;
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * p.nq / G;
  const int64_t q1 = static_cast<int64_t>(blockIdx.x + 1) * p.nq / G;
  if (q0 >= q1) return;
  if (threadIdx.x == 0) {
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L::bar_off);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&full[S + s], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x >= kConsumers)
    produce<VT, VW, S>(p, sm, q0, q1);
  else
    consume<VT, VW, S>(p, sm, q0, q1);
}

constexpr int kStages = 3;

template <typename VT, int VW>
maxe_status launch_variant(const Params& p, int sms, cudaStream_t st) {
  using L = Layout<VT, VW, kStages>;
  auto kern = spmm_chunk_kernel<VT, VW, kStages>;
  static int occ = -1;  // resident CTAs per SM for this variant
  if (occ < 0) {
    MAXE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::bytes)));
    int o = 0;
    MAXE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kThreads, L::bytes));
    occ = o > 0 ? o : 1;
  }
  const int64_t G = std::min<int64_t>(p.nq, static_cast<int64_t>(sms) * occ);
  kern<<<static_cast<unsigned>(G), kThreads, L::bytes, st>>>(p);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status launch_dtype(const Params& p, int vw, int sms, cudaStream_t st) {
  if (vw == 1) return launch_variant<VT, 1>(p, sms, st);
  if (vw == 2) return launch_variant<VT, 2>(p, sms, st);
  if constexpr (sizeof(typename Acc<VT>::T) == 4) {
    if (vw == 4) return launch_variant<VT, 4>(p, sms, st);
  }
  return MAXE_ERR_UNSUPPORTED;
}

}  // namespace

maxe_status spmv_build_partition(maxe_handle* h, cudaStream_t st) {
  const int64_t nq = std::max<int64_t>(1, ceil_div(h->nnz, kChunk));
  h->chunk_row = static_cast<int32_t*>(h->al.get(static_cast<size_t>(nq + 1) * sizeof(int32_t)));
  if (!h->chunk_row) return MAXE_ERR_OOM;
  h->nq = static_cast<int32_t>(nq);
  // chunk_row[q] = min{ r : rowptr[r+1] >= q*C + 1 }, then chunk 0 owns leading empty rows.
  MAXE_TRY(bucket_lower_bounds(h->rowptr + 1, h->rows, kChunk, 1, nq, h->chunk_row, st));
  MAXE_CUDA_TRY(cudaMemsetAsync(h->chunk_row, 0, sizeof(int32_t), st));
  return MAXE_OK;
}

maxe_status spmm_launch(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        const int32_t* yperm, cudaStream_t st) {
  if (h->rows == 0 || k == 0) return MAXE_OK;
  Params p{};
  p.rowptr = h->rowptr;
  p.col = h->col;
  p.val = h->val;
  p.X = X;
  p.Y = Y;
  p.yperm = yperm;
  p.chunk_row = h->chunk_row;
  p.status = h->status;
  p.ldx = ldx;
  p.ldy = ldy;
  p.Z = h->nnz;
  p.k = k;
  p.M = h->rows;
  p.nq = h->nq;
  const int eb = vector_bytes(h->dtype);
  auto aligned = [&](int vw) {
    const uintptr_t a = static_cast<uintptr_t>(vw) * eb;
    return ldx % vw == 0 && ldy % vw == 0 && reinterpret_cast<uintptr_t>(X) % a == 0 &&
           reinterpret_cast<uintptr_t>(Y) % a == 0;
  };
  int vw = 1;
  if (k > 1) {
    if (h->dtype != MAXE_F64 && k >= 3 && aligned(4))
      vw = 4;
    else if (aligned(2))
      vw = 2;
  }
  switch (h->dtype) {
    case MAXE_F64:
      return launch_dtype<double>(p, vw, h->sms, st);
    case MAXE_F32:
      return launch_dtype<float>(p, vw, h->sms, st);
    case MAXE_BF16:
      return launch_dtype<uint16_t>(p, vw, h->sms, st);
  }
  return MAXE_ERR_INVALID;
}

}  // namespace maxe
