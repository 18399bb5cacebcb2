// spmv_warp.cuh -- device side of the warp-per-row-chunk CSR SpMV/SpMM
// (Section 2 product on the permuted matrix of Eq. 1), shared by the
// single-matrix launch (spmv.cu) and the batched persistent launch (batch.cu).
// See spmv.cu for the design.
#pragma once

#include <climits>

#include "handle.cuh"

namespace maxe {
namespace warp {


constexpr int kWarps = 8;        // warps per block
constexpr int kThreads = kWarps * 32;
constexpr int kStages = 2;               // bulk-copy ring depth per warp
constexpr int kMaxItems = 16;            // consecutive entries per lane: 8 or 16 (tuned per handle)
constexpr int kMaxK = 64;

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
  const int32_t* wrow;
  unsigned* status;
  uint64_t wait_ns;  // limit of the bounded waits
  int64_t ldx, ldy;
  int32_t k, M, nW;
};

// X[c, c0 .. c0+VW) into xv.  A group past column k is read as a whole vector
// when the row is padded (ldx >= c0 + VW: still inside the row) and the unused
// lanes are zeroed; otherwise the tail columns are read one by one.
template <int VW, typename AT>
__device__ __forceinline__ void xload(const AT* __restrict__ X, int32_t c, int64_t ldx, int c0, int k, AT (&xv)[VW]) {
  const AT* px = X + static_cast<int64_t>(c) * ldx + c0;
  if constexpr (VW == 1) {
    xv[0] = __ldg(px);
  } else {
    if (c0 + VW <= k || c0 + VW <= ldx) {
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
      if (c0 + VW > k) {
#pragma unroll
        for (int w = 0; w < VW; ++w)
          if (c0 + w >= k) xv[w] = AT(0);
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

// Per-warp shared memory: an S-stage ring of COL/VAL pieces filled by 1-D bulk
// copies (TMA) with one mbarrier per stage, the row-start bitmap of the current
// piece, the scanned sums it is read back from, and the carries of the k columns.
// The mbarriers come first so that every variant keeps them at offset 0: a
// warp of the batched kernel runs ranges of different variants through the
// same ring and keeps its phase count across them.
template <typename VT, int VW, int IT>
struct alignas(16) WarpSmem {
  using AT = typename Acc<VT>::T;
  static constexpr int kPiece = 32 * IT;
  uint64_t full[kStages];
  int32_t col[kStages][kPiece];
  VT val[kStages][kPiece];
  AT sums[kPiece * VW];
  uint32_t flags[kPiece / 32];
  AT carry[kMaxK + 4];
};

template <typename VT, int VW, int IT>
constexpr size_t block_smem() {
  return sizeof(WarpSmem<VT, VW, IT>) * kWarps;
}

// A lane's N 16-byte words of a piece in shared memory, read without bank
// conflicts: lanes of one 8-lane access phase sit N words apart, so lane l
// starts at word (l*N/8) mod N and the loaded words are rotated back in
// registers (log2 N select stages).
template <int N>
__device__ __forceinline__ void lds_words(const uint4* base, uint4 (&w)[N], int lane) {
  const int rot = ((lane * N) >> 3) & (N - 1);
#pragma unroll
  for (int q = 0; q < N; ++q) w[q] = base[(q + rot) & (N - 1)];
#pragma unroll
  for (int bit = 1; bit < N; bit <<= 1) {
    if (rot & bit) {
      uint4 t[N];
#pragma unroll
      for (int i = 0; i < N; ++i) t[i] = w[(i - bit + N) & (N - 1)];
#pragma unroll
      for (int i = 0; i < N; ++i) w[i] = t[i];
    }
  }
}

template <int IT>
__device__ __forceinline__ void lds_cols(const int32_t* p, int32_t (&c)[IT], int lane) {
  uint4 w[IT / 4];
  lds_words<IT / 4>(reinterpret_cast<const uint4*>(p), w, lane);
#pragma unroll
  for (int i = 0; i < IT / 4; ++i) {
    c[4 * i] = static_cast<int32_t>(w[i].x), c[4 * i + 1] = static_cast<int32_t>(w[i].y);
    c[4 * i + 2] = static_cast<int32_t>(w[i].z), c[4 * i + 3] = static_cast<int32_t>(w[i].w);
  }
}

template <int IT>
__device__ __forceinline__ void lds_vals(const float* p, float (&a)[IT], int lane) {
  uint4 w[IT / 4];
  lds_words<IT / 4>(reinterpret_cast<const uint4*>(p), w, lane);
#pragma unroll
  for (int i = 0; i < IT / 4; ++i) {
    a[4 * i] = __uint_as_float(w[i].x), a[4 * i + 1] = __uint_as_float(w[i].y);
    a[4 * i + 2] = __uint_as_float(w[i].z), a[4 * i + 3] = __uint_as_float(w[i].w);
  }
}
template <int IT>
__device__ __forceinline__ void lds_vals(const double* p, double (&a)[IT], int lane) {
  uint4 w[IT / 2];
  lds_words<IT / 2>(reinterpret_cast<const uint4*>(p), w, lane);
#pragma unroll
  for (int i = 0; i < IT / 2; ++i) {
    a[2 * i] = __hiloint2double(static_cast<int>(w[i].y), static_cast<int>(w[i].x));
    a[2 * i + 1] = __hiloint2double(static_cast<int>(w[i].w), static_cast<int>(w[i].z));
  }
}
template <int IT>
__device__ __forceinline__ void lds_vals(const uint16_t* p, float (&a)[IT], int lane) {
  uint4 w[IT / 8];
  lds_words<IT / 8>(reinterpret_cast<const uint4*>(p), w, lane);
#pragma unroll
  for (int i = 0; i < IT / 8; ++i) {
    const uint32_t w4[4] = {w[i].x, w[i].y, w[i].z, w[i].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[8 * i + 2 * q] = __uint_as_float(w4[q] << 16);
      a[8 * i + 2 * q + 1] = __uint_as_float(w4[q] & 0xFFFF0000u);
    }
  }
}

__device__ __forceinline__ float to_acc_value(float v) { return v; }
__device__ __forceinline__ double to_acc_value(double v) { return v; }
__device__ __forceinline__ float to_acc_value(uint16_t v) { return __uint_as_float(static_cast<uint32_t>(v) << 16); }

// Scanned sums of a piece are stored transposed, entry e = IT*lane + j at slot
// (j*32 + lane): a warp's stores of one j are consecutive (conflict-free).
template <int IT, int VW>
__device__ __forceinline__ int sum_slot(int e) {
  return ((e % IT) * 32 + e / IT) * VW;
}

template <int VW, typename AT>
__device__ __forceinline__ void sts_vec(AT* p, const AT (&v)[VW]) {
  if constexpr (VW == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (VW == 2 && sizeof(AT) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (VW == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}

template <typename VT, int VW, int IT>
__device__ __forceinline__ void issue_piece(WarpSmem<VT, VW, IT>& ws, int s, const Params& p, int32_t base,
                                            uint64_t pol) {
  constexpr int kPiece = 32 * IT;
  mbar_arrive_expect_tx(&ws.full[s], kPiece * (4u + static_cast<uint32_t>(sizeof(VT))));
  bulk_g2s(ws.col[s], p.col + base, kPiece * 4u, &ws.full[s], pol);
  bulk_g2s(ws.val[s], static_cast<const VT*>(p.val) + base, kPiece * static_cast<uint32_t>(sizeof(VT)), &ws.full[s],
           pol);
}

// One kernel variant: value type VT, VW columns per pass, IT entries per lane;
// UNIT: k = 1 with unit strides (plain SpMV), so x and y are indexed directly.
// kMinBlocks: resident blocks per SM the register budget is cut for.
template <typename VT_, int VW_, int IT_, bool UNIT_>
struct Cfg {
  using VT = VT_;
  static constexpr int VW = VW_, IT = IT_;
  static constexpr bool UNIT = UNIT_;
  static constexpr int kMinBlocks =
      IT == 16 ? 2 : (sizeof(typename Acc<VT>::T) == 8 ? (VW == 1 ? 3 : 2) : (VW == 1 ? 4 : (VW == 2 ? 3 : 2)));
};

// Warp `w` of the partition in p.wrow: stream the entries of the rows it owns
// and write their outputs.  gi counts the pieces this warp has already taken
// through its ring (stage = gi % kStages, mbarrier parity = (gi / kStages) & 1),
// so one warp can run several ranges back to back (the batched kernel).
// Returns false if a bounded wait ran out.
template <class C>
__device__ __forceinline__ bool process_range(const Params& p, int32_t w, unsigned char* wsmem, uint32_t& gi) {
  using VT = typename C::VT;
  constexpr int VW = C::VW, IT = C::IT;
  constexpr bool UNIT = C::UNIT;
  using AT = typename Acc<VT>::T;
  constexpr int kItems = IT;
  constexpr int kPiece = 32 * IT;
  const int lane = threadIdx.x & 31;
  WarpSmem<VT, VW, IT>& ws = *reinterpret_cast<WarpSmem<VT, VW, IT>*>(wsmem);
  const AT* X = static_cast<const AT*>(p.X);
  AT* Y = static_cast<AT*>(p.Y);
  const int k = p.k;
  const int ngroups = (k + VW - 1) / VW;

  const int32_t r_hi = p.wrow[w + 1];
  int32_t r = p.wrow[w];  // first row of the range not yet written
  const int32_t e_lo = p.rowptr[r];
  const int32_t e_hi = p.rowptr[r_hi];
  const int32_t base0 = e_lo & ~7;  // 16-byte aligned for every value type
  const int32_t npieces = (e_hi > base0) ? (e_hi - base0 + kPiece - 1) / kPiece : 0;
  const uint64_t pol = policy_evict_first();
  for (int c = lane; c < ngroups * VW; c += 32) ws.carry[c] = AT(0);
  if (lane < kPiece / 32) ws.flags[lane] = 0u;
  __syncwarp();
  if (lane == 0)
    for (int s = 0; s < kStages && s < npieces; ++s)
      issue_piece(ws, static_cast<int>((gi + s) % kStages), p, base0 + s * kPiece, pol);

  int32_t r_start = e_lo;  // first entry of row r
  int32_t end0 = (r + lane < r_hi) ? __ldg(p.rowptr + r + 1 + lane) : INT_MAX;

  for (int32_t i = 0; i < npieces; ++i) {
    const uint32_t g = gi + static_cast<uint32_t>(i);
    const int s = static_cast<int>(g % kStages);
    const int32_t base = base0 + i * kPiece;
    // rows ending in this piece: flags in the bitmap, count, last end
    int nend = 0;
    int32_t last_o = -1;
    {
      int32_t end = end0;
      while (true) {
        const int32_t o = end - base;  // end <= INT_MAX and base >= 0: no overflow
        const bool in = o <= kPiece;
        const int n = __popc(__ballot_sync(0xffffffffu, in));
        if (in && o >= 1 && o < kPiece) atomicOr(&ws.flags[o >> 5], 1u << (o & 31));
        if (n > 0) last_o = __shfl_sync(0xffffffffu, o, n - 1);
        nend += n;
        if (n < 32) break;
        const int32_t rr = r + nend + lane;
        end = (rr < r_hi) ? __ldg(p.rowptr + rr + 1) : INT_MAX;
      }
    }
    const int32_t rn = r + nend;
    const int32_t end_first = end0;
    end0 = (rn + lane < r_hi) ? __ldg(p.rowptr + rn + 1 + lane) : INT_MAX;  // next piece, one step ahead
    __syncwarp();
    const uint32_t fw = (ws.flags[(kItems * lane) >> 5] >> ((kItems * lane) & 31)) & ((1u << kItems) - 1u);
    const int first_flag = fw ? __ffs(fw) - 1 : kItems;

    bool ok = mbar_wait_bounded(&ws.full[s], (g / kStages) & 1u, p.status, p.wait_ns);
    if (!__all_sync(0xffffffffu, ok)) return false;
    int32_t cj[kItems];
    AT a[kItems];
    lds_cols<IT>(ws.col[s] + kItems * lane, cj, lane);
    lds_vals<IT>(ws.val[s] + kItems * lane, a, lane);
    __syncwarp();
    if (lane < kPiece / 32) ws.flags[lane] = 0u;  // every lane has its flag bits
    // entries outside [e_lo, e_hi) belong to other warps (first and last piece only)
    uint32_t vmask = (1u << kItems) - 1u;
    if (!(base >= e_lo && base + kPiece <= e_hi)) {
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const int32_t e = base + kItems * lane + j;
        if (e < e_lo || e >= e_hi) vmask &= ~(1u << j);
      }
    }
    // the stage is in registers: refill it with piece i + kStages
    __syncwarp();
    if (lane == 0 && i + kStages < npieces) {
      fence_proxy_async_smem();
      issue_piece(ws, s, p, base + kStages * kPiece, pol);
    }

    for (int g = 0; g < ngroups; ++g) {
      const int c0 = g * VW;
      // products fused with the serial segmented scan over the lane's entries:
      // v[j] = a_j x_j + (j starts a row ? 0 : v[j-1])  -- one FMA per entry
      AT v[kItems][VW];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const bool head = j == 0 || ((fw >> j) & 1u);
        if ((vmask >> j) & 1u) {
          AT xv[VW];
          if constexpr (UNIT) {
            xv[0] = X[cj[j]];  // plain load: read-only-path loads here trip ptxas (C7600)
          } else {
            xload<VW>(X, cj[j], p.ldx, c0, k, xv);
          }
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] = head ? a[j] * xv[u] : fma(a[j], xv[u], v[j > 0 ? j - 1 : 0][u]);
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) v[j][u] = head ? AT(0) : v[j > 0 ? j - 1 : 0][u];
        }
      }
      int F = fw != 0u;
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
      const int Fe = __shfl_up_sync(0xffffffffu, F, 1);
      AT P[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const AT Ve = __shfl_up_sync(0xffffffffu, V[u], 1);
        const AT cin = ws.carry[c0 + u];
        P[u] = (lane == 0) ? cin : (Fe ? Ve : cin + Ve);
      }
#pragma unroll
      for (int j = 0; j < kItems; ++j) sts_vec<VW>(ws.sums + (j * 32 + lane) * VW, v[j]);
      // The prefix P belongs to the lane's leading segment [0, first_flag); the
      // only entry of it that is ever read (a row end, or the piece's carry) is
      // its last one, so P is added there alone.
      if (first_flag > 0) {
        AT* q = ws.sums + ((first_flag - 1) * 32 + lane) * VW;
#pragma unroll
        for (int u = 0; u < VW; ++u) q[u] += P[u];
      }
      __syncwarp();
      // rows that end in the piece
      int32_t prev_end = r_start;
      for (int b = 0; b < nend; b += 32) {
        const int32_t rr = r + b + lane;
        int32_t end = end_first;
        if (b > 0) end = (rr < r_hi) ? __ldg(p.rowptr + rr + 1) : INT_MAX;
        int32_t start = __shfl_up_sync(0xffffffffu, end, 1);
        if (lane == 0) start = prev_end;
        if (b + lane < nend) {
          AT out[VW];
          if (end > start) {
            const AT* src = ws.sums + sum_slot<IT, VW>(end - base - 1);
#pragma unroll
            for (int u = 0; u < VW; ++u) out[u] = src[u];
          } else {
#pragma unroll
            for (int u = 0; u < VW; ++u) out[u] = AT(0);
          }
          const int32_t row = p.yperm ? p.yperm[rr] : rr;
          if constexpr (UNIT)
            Y[row] = out[0];
          else
            ystore<VW>(Y, static_cast<int64_t>(row), p.ldy, c0, k, out);
        }
        prev_end = __shfl_sync(0xffffffffu, end, 31);
      }
      // partial row running on into the next piece
      if (lane < VW) ws.carry[c0 + lane] = (last_o == kPiece) ? AT(0) : ws.sums[sum_slot<IT, VW>(kPiece - 1) + lane];
      __syncwarp();
    }
    if (nend > 0) r_start = base + last_o;
    r = rn;
  }
  // rows left over are empty (their entries were all consumed)
  for (int32_t rr = r + lane; rr < r_hi; rr += 32) {
    const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
    for (int c = 0; c < k; ++c) Y[row * p.ldy + c] = AT(0);
  }
  gi += static_cast<uint32_t>(npieces);
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// SpMM with lanes over columns (k >= 5 for FP32 values, k >= 3 for FP64).
//
// The warp splits into G = 32/g groups of g lanes; lane `sub` of a group owns
// VC = 4 (FP32) or 2 (FP64) consecutive columns, so a group covers CB = g*VC
// columns (blocks of CB columns are processed one after the other).  Group q
// walks its chunk of C = 256/G consecutive entries of the piece in order,
// accumulating with FMAs: the X row of an entry is one coalesced load per group
// (one L2 request instead of one per 4 columns), and a row that starts and ends
// inside the chunk is complete in registers and written at once.  Only the
// first segment of each chunk (the row running in from the previous chunk) and
// the tail go through a segmented scan across the G groups (log2 G shuffle
// steps), as in the single-column kernel.  Rows are found by their end offset
// (first row of the piece with rowptr[r+1] >= base + o).
// Ring of the column-lanes kernel: each 32-entry segment of a piece is
// followed by 16 bytes of padding, so the chunks that the groups read at the
// same time fall into different shared-memory banks.  (The mbarriers stay at
// offset 0, as in WarpSmem.)
template <typename VT>
struct alignas(16) WarpSmemLC {
  using AT = typename Acc<VT>::T;
  static constexpr int kPiece = 256, kSegs = kPiece / 32;
  static constexpr int kColStride = 32 + 4;                                  // int32 per segment
  static constexpr int kValStride = 32 + 16 / static_cast<int>(sizeof(VT));  // values per segment
  uint64_t full[kStages];
  int32_t col[kStages][kSegs * kColStride];
  VT val[kStages][kSegs * kValStride];
  uint32_t flags[kPiece / 32];
  AT carry[kMaxK + 4];
  __device__ __forceinline__ int32_t c(int s, int e) const { return col[s][(e >> 5) * kColStride + (e & 31)]; }
  __device__ __forceinline__ VT v(int s, int e) const { return val[s][(e >> 5) * kValStride + (e & 31)]; }
};

// One bulk copy per 32-entry segment and array, issued by lanes 0..15.
template <typename VT>
__device__ __forceinline__ void issue_piece_lc(WarpSmemLC<VT>& ws, int s, const Params& p, int32_t base,
                                               uint64_t pol) {
  using WS = WarpSmemLC<VT>;
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_arrive_expect_tx(&ws.full[s], WS::kPiece * (4u + static_cast<uint32_t>(sizeof(VT))));
  __syncwarp();
  if (lane < WS::kSegs) {
    bulk_g2s(&ws.col[s][lane * WS::kColStride], p.col + base + 32 * lane, 32 * 4u, &ws.full[s], pol);
  } else if (lane < 2 * WS::kSegs) {
    const int j = lane - WS::kSegs;
    bulk_g2s(&ws.val[s][j * WS::kValStride], static_cast<const VT*>(p.val) + base + 32 * j,
             32 * static_cast<uint32_t>(sizeof(VT)), &ws.full[s], pol);
  }
}

template <typename VT>
__device__ __forceinline__ int32_t row_ending_at(const Params& p, int32_t lo, int32_t hi, int32_t target) {
  while (lo < hi) {  // first row in [lo, hi] whose end >= target
    const int32_t mid = (lo + hi) >> 1;
    if (__ldg(p.rowptr + mid + 1) >= target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

template <typename VT>
__device__ __forceinline__ bool process_range_lc(const Params& p, int32_t w, unsigned char* wsmem, uint32_t& gi,
                                                 int g) {
  using AT = typename Acc<VT>::T;
  constexpr int IT = 8;
  constexpr int kPiece = 32 * IT;
  constexpr int VC = sizeof(AT) == 4 ? 4 : 2;
  const int lane = threadIdx.x & 31;
  WarpSmemLC<VT>& ws = *reinterpret_cast<WarpSmemLC<VT>*>(wsmem);
  const AT* X = static_cast<const AT*>(p.X);
  AT* Y = static_cast<AT*>(p.Y);
  const int k = p.k;
  const int G = 32 / g, C = kPiece / G;
  const int q = lane / g, sub = lane - q * g;
  const int CB = g * VC;
  const int nblocks = (k + CB - 1) / CB;

  const int32_t r_hi = p.wrow[w + 1];
  int32_t r = p.wrow[w];
  const int32_t e_lo = p.rowptr[r];
  const int32_t e_hi = p.rowptr[r_hi];
  const int32_t base0 = e_lo & ~7;
  const int32_t npieces = (e_hi > base0) ? (e_hi - base0 + kPiece - 1) / kPiece : 0;
  const uint64_t pol = policy_evict_first();
  for (int c = lane; c < nblocks * CB; c += 32) ws.carry[c] = AT(0);
  if (lane < kPiece / 32) ws.flags[lane] = 0u;
  __syncwarp();
  for (int s = 0; s < kStages && s < npieces; ++s)
    issue_piece_lc(ws, static_cast<int>((gi + s) % kStages), p, base0 + s * kPiece, pol);

  int32_t r_start = e_lo;
  int32_t end0 = (r + lane < r_hi) ? __ldg(p.rowptr + r + 1 + lane) : INT_MAX;

  for (int32_t i = 0; i < npieces; ++i) {
    const uint32_t gg = gi + static_cast<uint32_t>(i);
    const int s = static_cast<int>(gg % kStages);
    const int32_t base = base0 + i * kPiece;
    int nend = 0;
    int32_t last_o = -1;
    {
      int32_t end = end0;
      while (true) {
        const int32_t o = end - base;
        const bool in = o <= kPiece;
        const int n = __popc(__ballot_sync(0xffffffffu, in));
        if (in && o >= 1 && o < kPiece) atomicOr(&ws.flags[o >> 5], 1u << (o & 31));
        if (n > 0) last_o = __shfl_sync(0xffffffffu, o, n - 1);
        nend += n;
        if (n < 32) break;
        const int32_t rr = r + nend + lane;
        end = (rr < r_hi) ? __ldg(p.rowptr + rr + 1) : INT_MAX;
      }
    }
    const int32_t rn = r + nend;
    const int32_t end_first = end0;
    end0 = (rn + lane < r_hi) ? __ldg(p.rowptr + rn + 1 + lane) : INT_MAX;
    __syncwarp();
    const int e0 = q * C;  // the group's chunk, piece-relative
    const uint32_t wa = ws.flags[e0 >> 5];
    const uint32_t wb = ws.flags[min((e0 + C - 1) >> 5, kPiece / 32 - 1)];
    bool ok = mbar_wait_bounded(&ws.full[s], (gg / kStages) & 1u, p.status, p.wait_ns);
    if (!__all_sync(0xffffffffu, ok)) return false;
    __syncwarp();
    if (lane < kPiece / 32) ws.flags[lane] = 0u;
    const int32_t rlast = rn - 1;  // rows ending in the piece: [r, rn)

    for (int blk = 0; blk < nblocks; ++blk) {
      const int cs = blk * CB + sub * VC;  // the lane's first column
      AT acc[VC], head[VC];
#pragma unroll
      for (int u = 0; u < VC; ++u) acc[u] = head[u] = AT(0);
      bool seen = false;
      int ffe = 0;           // first row end in the chunk (piece-relative)
      int32_t rcur = r - 1;  // last row completed inside the chunk
      for (int i0 = 0; i0 < C; i0 += 8) {
        AT xv[8][VC];
        AT av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + i0 + u;
          const int32_t ge = base + e;
          av[u] = AT(0);
#pragma unroll
          for (int c = 0; c < VC; ++c) xv[u][c] = AT(0);
          if (ge >= e_lo && ge < e_hi) {
            av[u] = to_acc_value(ws.v(s, e));
            xload<VC>(X, ws.c(s, e), p.ldx, cs, k, xv[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + i0 + u;
          const uint32_t word = ((e >> 5) == (e0 >> 5)) ? wa : wb;
          if ((word >> (e & 31)) & 1u) {  // a row ends at e: [.., e) is complete
            if (!seen) {
              seen = true;
              ffe = e;
#pragma unroll
              for (int c = 0; c < VC; ++c) head[c] = acc[c];
            } else {
              int32_t rr = rcur + 1;
              if (rcur < r) rr = row_ending_at<VT>(p, r, rlast, base + e);
              while (__ldg(p.rowptr + rr + 1) < base + e) ++rr;  // skip empty rows
              rcur = rr;
              const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
              ystore<VC>(Y, row, p.ldy, cs, k, acc);
            }
#pragma unroll
            for (int c = 0; c < VC; ++c) acc[c] = AT(0);
          }
#pragma unroll
          for (int c = 0; c < VC; ++c) acc[c] = fma(av[u], xv[u][c], acc[c]);
        }
      }
      if (!seen) {
#pragma unroll
        for (int c = 0; c < VC; ++c) head[c] = AT(0);
      }
      // segmented scan of (seen, tail) across the groups
      int F = seen;
      AT V[VC];
#pragma unroll
      for (int c = 0; c < VC; ++c) V[c] = acc[c];
      for (int d = 1; d < G; d <<= 1) {
        const int Fu = __shfl_up_sync(0xffffffffu, F, d * g);
        AT Vu[VC];
#pragma unroll
        for (int c = 0; c < VC; ++c) Vu[c] = __shfl_up_sync(0xffffffffu, V[c], d * g);
        if (q >= d) {
          if (!F)
#pragma unroll
            for (int c = 0; c < VC; ++c) V[c] += Vu[c];
          F |= Fu;
        }
      }
      const int Fe = __shfl_up_sync(0xffffffffu, F, g);
      AT P[VC], cin[VC];
#pragma unroll
      for (int c = 0; c < VC; ++c) {
        const AT Ve = __shfl_up_sync(0xffffffffu, V[c], g);
        cin[c] = (cs + c < kMaxK + 4) ? ws.carry[cs + c] : AT(0);
        P[c] = (q == 0) ? cin[c] : (Fe ? Ve : cin[c] + Ve);
      }
      if (seen) {  // the row running into the chunk ends at its first row end
        const int32_t rr = row_ending_at<VT>(p, r, rlast, base + ffe);
        AT out[VC];
#pragma unroll
        for (int c = 0; c < VC; ++c) out[c] = P[c] + head[c];
        const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
        ystore<VC>(Y, row, p.ldy, cs, k, out);
      }
      // inclusive value of the last group, per column of this lane
      const int src = (G - 1) * g + sub;
      const int Fl = __shfl_sync(0xffffffffu, F, src);
      AT inc[VC];
#pragma unroll
      for (int c = 0; c < VC; ++c) {
        const AT Vl = __shfl_sync(0xffffffffu, V[c], src);
        inc[c] = Fl ? Vl : cin[c] + Vl;
      }
      __syncwarp();
      if (last_o == kPiece) {  // a row ends exactly at the end of the piece
        if (q == G - 1) {
          const int32_t rr = row_ending_at<VT>(p, r, rlast, base + kPiece);
          const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
          ystore<VC>(Y, row, p.ldy, cs, k, inc);
        }
        if (q == 0)
#pragma unroll
          for (int c = 0; c < VC; ++c)
            if (cs + c < kMaxK + 4) ws.carry[cs + c] = AT(0);
      } else if (q == 0) {
#pragma unroll
        for (int c = 0; c < VC; ++c)
          if (cs + c < kMaxK + 4) ws.carry[cs + c] = inc[c];
      }
      __syncwarp();
    }
    // empty rows of the piece get zeros
    int32_t prev_end = r_start;
    for (int b = 0; b < nend; b += 32) {
      const int32_t rr = r + b + lane;
      int32_t end = end_first;
      if (b > 0) end = (rr < r_hi) ? __ldg(p.rowptr + rr + 1) : INT_MAX;
      int32_t start = __shfl_up_sync(0xffffffffu, end, 1);
      if (lane == 0) start = prev_end;
      if (b + lane < nend && end == start) {
        const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
        for (int c = 0; c < k; ++c) Y[row * p.ldy + c] = AT(0);
      }
      prev_end = __shfl_sync(0xffffffffu, end, 31);
    }
    if (nend > 0) r_start = base + last_o;
    r = rn;
    // the stage has been read: refill it with piece i + kStages
    __syncwarp();
    if (i + kStages < npieces) {
      fence_proxy_async_smem();
      issue_piece_lc(ws, s, p, base + kStages * kPiece, pol);
    }
  }
  for (int32_t rr = r + lane; rr < r_hi; rr += 32) {
    const int64_t row = p.yperm ? static_cast<int64_t>(p.yperm[rr]) : static_cast<int64_t>(rr);
    for (int c = 0; c < k; ++c) Y[row * p.ldy + c] = AT(0);
  }
  gi += static_cast<uint32_t>(npieces);
  __syncwarp();
  return true;
}

// groups of g lanes for k columns (0: use the column-pass kernel instead)
__host__ __device__ inline int lc_group(int k, int value_bytes_acc, int ldx, int ldy) {
  const int vc = value_bytes_acc == 4 ? 4 : 2;
  if (k < (vc == 4 ? 5 : 3) || ldx % vc != 0 || ldy % vc != 0) return 0;
  if (k <= 2 * vc) return 2;
  if (k <= 4 * vc) return 4;
  return 8;
}

template <typename VT>
__global__ void __launch_bounds__(kThreads, 2) spmm_lc_kernel(Params p, int g) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarps + wib;
  if (w >= p.nW) return;
  unsigned char* wsmem = smem_raw + sizeof(WarpSmemLC<VT>) * wib;
  WarpSmemLC<VT>& ws = *reinterpret_cast<WarpSmemLC<VT>*>(wsmem);
  if ((threadIdx.x & 31) == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&ws.full[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t gi = 0;
  process_range_lc<VT>(p, w, wsmem, gi, g);
}

template <class C>
__device__ __forceinline__ void init_ring(unsigned char* wsmem) {
  using WS = WarpSmem<typename C::VT, C::VW, C::IT>;
  WS& ws = *reinterpret_cast<WS*>(wsmem);
  if ((threadIdx.x & 31) == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&ws.full[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
}

template <class C>
__global__ void __launch_bounds__(kThreads, C::kMinBlocks) spmm_warp_kernel(Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarps + wib;
  if (w >= p.nW) return;
  unsigned char* wsmem = smem_raw + sizeof(WarpSmem<typename C::VT, C::VW, C::IT>) * wib;
  init_ring<C>(wsmem);
  uint32_t gi = 0;
  process_range<C>(p, w, wsmem, gi);
}


}  // namespace warp
}  // namespace maxe
