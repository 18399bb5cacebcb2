// coo.cu -- SpMV over the COO form of the permuted matrix (Section 2: triplets
// (ROW, COL, VALUE), 3 x nnz storage).  The handle's COO shares COL and VALUE
// with its CSR and adds ROW, so the triplets are row-sorted; the product is
// deterministic.
//
// Work split: chunks of 256 consecutive entries, one warp per chunk, 8 entries
// per lane -- nnz-balanced by construction, whatever the row lengths.  ROW, COL
// and VALUE are streamed with 16-byte loads that bypass L1 and are evicted
// first from L2, so the x gathers keep the cache.
//
// Inside a chunk (rows are non-decreasing):
//   - each lane sums its own segments; a segment that starts and ends inside
//     the lane is a whole row and is written at once;
//   - the lanes' last segments are combined by a segmented shuffle scan; a
//     lane's first segment adds the scan value of the lane before it when
//     they share the row;
//   - a segment holding the chunk's first row is a whole row only if that row
//     starts in this chunk, and one holding its last row only if the row ends
//     in it.  Otherwise the chunk's partial sums go to per-chunk carries
//     (head, tail) and a second kernel adds them up, in chunk order, for every
//     row that crosses a chunk boundary.
//   - Rows with no entries are written as zeros by the lane holding the next
//     row's first entry (and the last entry zeroes the rows after it); runs of
//     more than 32 empty rows by the whole warp.
#include <algorithm>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kItems = 8;
constexpr int kChunk = 32 * kItems;  // entries per warp
constexpr int kWarps = 8;
constexpr uint8_t kHead = 1, kTail = 2, kPass = 4;

__global__ void coo_rows_kernel(const int32_t* __restrict__ rowptr, int32_t M, int64_t Z, int32_t* __restrict__ row) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= Z) return;
  int32_t lo = 0, hi = M;  // last i with rowptr[i] <= e
  while (hi - lo > 1) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (rowptr[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  row[e] = lo;
}

template <typename V>
struct Vals;
template <>
struct Vals<double> {
  static __device__ __forceinline__ void load(const void* val, int64_t e, bool full, int64_t Z, double (&v)[kItems]) {
    const double* p = static_cast<const double*>(val) + e;
    if (full) {
#pragma unroll
      for (int q = 0; q < kItems / 2; ++q) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p) + q);
        v[2 * q] = t.x;
        v[2 * q + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kItems; ++j) v[j] = e + j < Z ? p[j] : 0.0;
    }
  }
};

struct ValsF32 {
  static __device__ __forceinline__ void load(const void* val, int64_t e, bool full, int64_t Z, float (&v)[kItems]) {
    const float* p = static_cast<const float*>(val) + e;
    if (full) {
#pragma unroll
      for (int q = 0; q < kItems / 4; ++q) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(p) + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kItems; ++j) v[j] = e + j < Z ? p[j] : 0.0f;
    }
  }
};

struct ValsBF16 {
  static __device__ __forceinline__ float up(uint32_t bits16) { return __uint_as_float(bits16 << 16); }
  static __device__ __forceinline__ void load(const void* val, int64_t e, bool full, int64_t Z, float (&v)[kItems]) {
    const uint16_t* p = static_cast<const uint16_t*>(val) + e;
    if (full) {
      const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
      const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[2 * q] = up(w[q] & 0xffffu);
        v[2 * q + 1] = up(w[q] >> 16);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kItems; ++j) v[j] = e + j < Z ? up(p[j]) : 0.0f;
    }
  }
};

template <typename VT>
__device__ __forceinline__ void put(VT* __restrict__ y, const int32_t* __restrict__ yperm, int32_t r, VT v) {
  y[yperm ? yperm[r] : r] = v;
}

template <typename VT>
__device__ __forceinline__ void zero_rows(VT* __restrict__ y, const int32_t* __restrict__ yperm, int32_t a,
                                          int32_t b) {
  for (int32_t r = a; r < b; ++r) put(y, yperm, r, VT(0));
}

// One warp per 256-entry chunk.  head/tail carries and flags per chunk.
template <typename VT, typename VL>
__global__ void __launch_bounds__(32 * kWarps) coo_spmv_kernel(const int32_t* __restrict__ row,
                                                               const int32_t* __restrict__ col,
                                                               const void* __restrict__ val, int64_t Z, int32_t M,
                                                               int64_t nch, const VT* __restrict__ x,
                                                               VT* __restrict__ y, const int32_t* __restrict__ yperm,
                                                               VT* __restrict__ carry_head, VT* __restrict__ carry_tail,
                                                               uint8_t* __restrict__ cflags) {
  const int lane = threadIdx.x & 31;
  const int64_t c = static_cast<int64_t>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
  if (c >= nch) return;
  const int64_t cb = c * kChunk, ce = std::min<int64_t>(cb + kChunk, Z);
  const int64_t e0 = cb + lane * kItems;
  const bool full = e0 + kItems <= Z;
  int32_t r[kItems], cj[kItems];
  if (full) {
#pragma unroll
    for (int q = 0; q < kItems / 4; ++q) {
      const int4 a = __ldcs(reinterpret_cast<const int4*>(row + e0) + q);
      const int4 b = __ldcs(reinterpret_cast<const int4*>(col + e0) + q);
      r[4 * q] = a.x, r[4 * q + 1] = a.y, r[4 * q + 2] = a.z, r[4 * q + 3] = a.w;
      cj[4 * q] = b.x, cj[4 * q + 1] = b.y, cj[4 * q + 2] = b.z, cj[4 * q + 3] = b.w;
    }
  } else {
    // entries past the end belong to a sentinel row M that is never written
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const bool ok = e0 + j < Z;
      r[j] = ok ? row[e0 + j] : M;
      cj[j] = ok ? col[e0 + j] : 0;
    }
  }
  VT p[kItems];
  VL::load(val, e0, full, Z, p);
#pragma unroll
  for (int j = 0; j < kItems; ++j) p[j] = (e0 + j < Z) ? p[j] * x[cj[j]] : VT(0);

  // rows of the chunk's first and last entries, and whether they cross its edges
  const int32_t r0 = row[cb], rl = row[ce - 1];
  const int last_lane = static_cast<int>((ce - 1 - cb) / kItems);
  const bool cont_in = cb > 0 && row[cb - 1] == r0;
  const bool cont_out = ce < Z && row[ce] == rl;

  // empty rows before each row start (and after the last entry)
  int32_t prev = __shfl_up_sync(0xffffffffu, r[kItems - 1], 1);
  if (lane == 0) prev = cb > 0 ? row[cb - 1] : -1;
  // a gap of up to 32 rows is written by its lane; a longer one by the whole warp
#pragma unroll
  for (int j = 0; j <= kItems; ++j) {
    int32_t ga = 0, gb = 0;
    if (j < kItems) {
      const int32_t pr = j == 0 ? prev : r[j - 1];
      if (e0 + j < Z && r[j] != pr) ga = pr + 1, gb = r[j];
    } else if (e0 <= Z - 1 && Z - 1 < e0 + kItems) {  // the rows after the last entry
      ga = row[Z - 1] + 1, gb = M;
    }
    if (gb - ga <= 32) zero_rows(y, yperm, ga, gb);
    for (unsigned m = __ballot_sync(0xffffffffu, gb - ga > 32); m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const int32_t a = __shfl_sync(0xffffffffu, ga, src), b = __shfl_sync(0xffffffffu, gb, src);
      for (int32_t q = a + lane; q < b; q += 32) put(y, yperm, q, VT(0));
    }
  }

  // lane-local segments: first (head), middle (whole rows), last (tail)
  VT acc = VT(0), hd = VT(0);
  bool single = true;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    acc += p[j];
    if (j + 1 < kItems && r[j + 1] != r[j]) {
      if (single)
        hd = acc;  // the lane's first segment, finished below
      else if (r[j] < M)
        put(y, yperm, r[j], acc);  // bounded on both sides inside the lane: a whole row
      single = false;
      acc = VT(0);
    }
  }
  const int32_t F = r[0], R = r[kItems - 1];
  // segmented inclusive scan of the tails: a lane starts a new segment unless it
  // is one segment continuing the previous lane's last row
  const int32_t Rprev = __shfl_up_sync(0xffffffffu, R, 1);
  int flag = (lane == 0 || !single || Rprev != R) ? 1 : 0;
  VT S = acc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const VT s_up = __shfl_up_sync(0xffffffffu, S, d);
    const int f_up = __shfl_up_sync(0xffffffffu, flag, d);
    if (lane >= d && !flag) S += s_up;
    if (lane >= d) flag |= f_up;
  }
  const VT Sprev = __shfl_up_sync(0xffffffffu, S, 1);
  const int32_t Fnext = __shfl_down_sync(0xffffffffu, F, 1);

  if (!single) {  // the lane's first segment ends inside the lane
    const VT v = hd + ((lane > 0 && Rprev == F) ? Sprev : VT(0));
    if (F == r0 && cont_in)
      carry_head[c] = v;
    else if (F < M)
      put(y, yperm, F, v);
  }
  if (lane < last_lane) {  // the tail ends here if the next lane starts a new row
    if (Fnext != R) {
      if (R == r0 && cont_in)
        carry_head[c] = S;
      else if (R < M)
        put(y, yperm, R, S);
    }
  } else if (lane == last_lane) {
    const bool pass = cont_in && cont_out && rl == r0;
    // R != rl only in a lane cut by the end of the matrix: its tail is the
    // sentinel row and row rl was finished inside the lane above
    if (R == rl) {
      if (pass || (!cont_out && rl == r0 && cont_in))
        carry_head[c] = S;  // the whole chunk is one row that started before it
      else if (cont_out)
        carry_tail[c] = S;
      else
        put(y, yperm, rl, S);
    }
    cflags[c] = static_cast<uint8_t>((cont_in ? kHead : 0) | (cont_out && !pass ? kTail : 0) | (pass ? kPass : 0));
  }
}

// Rows that cross chunk edges: the chunk where the row starts adds its tail and
// the following chunks' heads, in chunk order.
template <typename VT>
__global__ void coo_fixup_kernel(const int32_t* __restrict__ row, int64_t Z, int64_t nch,
                                 const VT* __restrict__ carry_head, const VT* __restrict__ carry_tail,
                                 const uint8_t* __restrict__ cflags, VT* __restrict__ y,
                                 const int32_t* __restrict__ yperm) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= nch || !(cflags[c] & kTail)) return;
  const int32_t r = row[std::min<int64_t>((c + 1) * kChunk, Z) - 1];
  VT s = carry_tail[c];
  for (int64_t d = c + 1; d < nch; ++d) {
    s += carry_head[d];
    if (!(cflags[d] & kPass)) break;
  }
  put(y, yperm, r, s);
}

template <typename VT>
__global__ void zero_kernel(VT* __restrict__ y, int32_t M) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < M) y[i] = VT(0);
}

template <typename VT, typename VL>
maxe_status run(const maxe_handle* h, const VT* x, VT* y, const int32_t* yperm, cudaStream_t st) {
  const int64_t Z = h->nnz;
  if (h->rows == 0) return MAXE_OK;
  if (Z == 0) {
    zero_kernel<VT><<<static_cast<unsigned>(ceil_div(h->rows, 256)), 256, 0, st>>>(y, h->rows);
    MAXE_CUDA_TRY(cudaGetLastError());
    return MAXE_OK;
  }
  const int64_t nch = ceil_div(Z, kChunk);
  VT* ch = static_cast<VT*>(h->coo_carry);
  uint8_t* cf = reinterpret_cast<uint8_t*>(ch + 2 * nch);
  coo_spmv_kernel<VT, VL><<<static_cast<unsigned>(ceil_div(nch, kWarps)), 32 * kWarps, 0, st>>>(
      h->coo_row, h->col, h->val, Z, h->rows, nch, x, y, yperm, ch, ch + nch, cf);
  MAXE_CUDA_TRY(cudaGetLastError());
  coo_fixup_kernel<VT><<<static_cast<unsigned>(ceil_div(nch, 256)), 256, 0, st>>>(h->coo_row, Z, nch, ch, ch + nch,
                                                                                   cf, y, yperm);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace

maxe_status coo_build(maxe_handle* h, cudaStream_t st) {
  const int64_t Z = h->nnz;
  const int64_t nch = ceil_div(std::max<int64_t>(Z, 1), kChunk);
  h->coo_row = static_cast<int32_t*>(h->al.get(static_cast<size_t>(std::max<int64_t>(Z, 1)) * sizeof(int32_t)));
  // carries: head[nch], tail[nch] of the vector type, then nch flag bytes
  h->coo_carry = h->al.get(static_cast<size_t>(nch) * (2 * vector_bytes(h->dtype) + 1));
  if (!h->coo_row || !h->coo_carry) return MAXE_ERR_OOM;
  if (Z > 0) {
    coo_rows_kernel<<<static_cast<unsigned>(ceil_div(Z, 256)), 256, 0, st>>>(h->rowptr, h->rows, Z, h->coo_row);
    MAXE_CUDA_TRY(cudaGetLastError());
  }
  return MAXE_OK;
}

maxe_status coo_spmv_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st) {
  if (h->dtype == MAXE_F64)
    return run<double, Vals<double>>(h, static_cast<const double*>(x), static_cast<double*>(y), yperm, st);
  if (h->dtype == MAXE_F32)
    return run<float, ValsF32>(h, static_cast<const float*>(x), static_cast<float*>(y), yperm, st);
  return run<float, ValsBF16>(h, static_cast<const float*>(x), static_cast<float*>(y), yperm, st);
}

}  // namespace maxe
