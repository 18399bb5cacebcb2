// spmm_rows.cuh -- the per-warp machinery of SpMM with one CSR row per group
// of lanes (Section 2's CSR product, k right-hand sides), shared by the
// single-matrix kernel (spmm_rows.cu) and the batched one (batch.cu).
//
// A warp works through a range of rows in chunks (at most kChunkR rows and
// kChunkE entries): stage_chunk copies a chunk's column indices and values
// into one half of the warp's double buffer (16-byte cp.async copies rounded
// out to 8-entry boundaries; the CSR arrays are padded past nnz) and writes its
// row pointers; rows_chunk multiplies the rows of a staged chunk, a group of G
// lanes per row, each lane a 16-byte piece of the X and Y rows (VC = 4 FP32 or
// 2 FP64 columns), gathering X pieces by the staged column indices and
// accumulating in registers.  Entries go eight at a time, their X loads issued
// together, into four partial sums (entries u and u + 4 of a step share one)
// added in a fixed order, so a Y row is one group's sum in a fixed order: the
// same bits whichever warp, launch or batch computes it.  A row longer than
// kChunkE is a chunk of its own; its entries past the staged ones are read
// from global memory.
#pragma once

#include "handle.cuh"

namespace maxe {
namespace rows {

constexpr int kRowsUnroll = 8;  // entries per step of a group
constexpr int kRowsParts = 4;   // partial sums of a group
constexpr int kChunkE = 256;    // entries of a chunk (a longer row: the first kChunkE)
constexpr int kChunkR = 63;     // rows of a chunk: its 64 row pointers are two per lane
constexpr int kSlotE = kChunkE + 8;  // staged slots: the chunk rounded out to 8-entry boundaries

template <typename VT>
struct RowsT;
template <>
struct RowsT<float> {
  using AT = float;
  using V = float4;
  static constexpr int VC = 4;
  static __device__ __forceinline__ float acc(float v) { return v; }
};
template <>
struct RowsT<uint16_t> {
  using AT = float;
  using V = float4;
  static constexpr int VC = 4;
  static __device__ __forceinline__ float acc(uint16_t v) { return __uint_as_float(static_cast<uint32_t>(v) << 16); }
};
template <>
struct RowsT<double> {
  using AT = double;
  using V = double2;
  static constexpr int VC = 2;
  static __device__ __forceinline__ double acc(double v) { return v; }
};

__device__ __forceinline__ void fma_vec(float4& acc, float a, const float4& x) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  acc.z = fmaf(a, x.z, acc.z);
  acc.w = fmaf(a, x.w, acc.w);
}
__device__ __forceinline__ void fma_vec(double2& acc, double a, const double2& x) {
  acc.x = fma(a, x.x, acc.x);
  acc.y = fma(a, x.y, acc.y);
}
__device__ __forceinline__ void add_vec(float4& a, const float4& b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}
__device__ __forceinline__ void add_vec(double2& a, const double2& b) {
  a.x += b.x;
  a.y += b.y;
}
// Y piece of a row: all VC columns, or the first `left` of them (the row's last piece)
__device__ __forceinline__ void store_piece(float4* y, const float4& v, int left) {
  if (left >= 4) {
    *y = v;
    return;
  }
  float* f = reinterpret_cast<float*>(y);
  f[0] = v.x;
  if (left > 1) f[1] = v.y;
  if (left > 2) f[2] = v.z;
}
__device__ __forceinline__ void store_piece(double2* y, const double2& v, int left) {
  if (left >= 2) {
    *y = v;
    return;
  }
  reinterpret_cast<double*>(y)[0] = v.x;
}
__device__ __forceinline__ void zero(float4& v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero(double2& v) { v = make_double2(0.0, 0.0); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One warp's double buffer: column indices, values and row pointers (slots
// relative to e0a) and extents of two chunks.
template <typename VT>
struct alignas(16) RowsStage {
  int32_t col[2][kSlotE];
  VT val[2][kSlotE];
  int32_t rp[2][kChunkR + 1];
  int64_t e0a[2];  // the chunk's first staged entry (a multiple of 8)
  int32_t r[2];    // its first row
  int32_t n[2];    // its rows
  int32_t lim[2];  // end of its staged slots: rows reaching past it are long rows
};

// The product a warp works on: Y' = A' X' with A' in CSR.
struct RowsOperand {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  const void* X;
  void* Y;
  const int32_t* yperm;  // Y row of row r: yperm[r] (null: r)
  int64_t ldx, ldy;
  int32_t k;
  int32_t pf;  // 1: prefetch the X rows of a group's next row into L2 (stencil-like matrices)
};

// Row pointers rowptr[r + j], j = 0 .. min(kChunkR, b - r): j = lane in *pa,
// j = 32 + lane in *pb; INT32_MAX past the warp's rows.
__device__ __forceinline__ void load_rp(const int32_t* rowptr, int32_t r, int32_t b, int lane, int32_t* pa,
                                        int32_t* pb) {
  const int32_t lim = min(kChunkR, b - r);
  *pa = lane <= lim ? __ldg(rowptr + r + lane) : INT32_MAX;
  *pb = 32 + lane <= lim ? __ldg(rowptr + r + 32 + lane) : INT32_MAX;
}

// Cuts the chunk that starts at row r (its row pointers in pa / pb): the most
// rows, up to kChunkR, whose entries fit in kChunkE, at least one row.  Stages
// its column indices and values into buffer `buf` (cp.async, committed) and
// writes its row pointers and extent; returns its row count.  Warp-uniform; all
// 32 lanes take part.
template <typename VT>
__device__ __forceinline__ int32_t stage_chunk(RowsStage<VT>* s, int buf, const RowsOperand& p, int32_t r, int32_t b,
                                               int lane, int32_t pa, int32_t pb) {
  const int32_t rows = min(kChunkR, b - r);
  const int32_t E0 = __shfl_sync(0xffffffffu, pa, 0);
  const bool oka = lane >= 1 && lane <= rows && pa - E0 <= kChunkE;
  const bool okb = 32 + lane <= rows && pb - E0 <= kChunkE;
  int32_t n = __popc(__ballot_sync(0xffffffffu, oka)) + __popc(__ballot_sync(0xffffffffu, okb));
  n = max(n, 1);
  const int32_t ea = __shfl_sync(0xffffffffu, pa, n & 31), eb = __shfl_sync(0xffffffffu, pb, n & 31);
  const int32_t E1 = n < 32 ? ea : eb;
  const int64_t e0a = static_cast<int64_t>(E0) & ~int64_t(7);
  const int32_t lim = static_cast<int32_t>(std::min<int64_t>(E1, static_cast<int64_t>(E0) + kChunkE) - e0a);
  const int32_t slots = (lim + 7) & ~7;  // <= kSlotE
  const int32_t* gcol = p.col + e0a;
  for (int i = lane; i < slots / 4; i += 32) cp_async16(&s->col[buf][4 * i], gcol + 4 * i);
  constexpr int per = 16 / static_cast<int>(sizeof(VT));
  const VT* gval = static_cast<const VT*>(p.val) + e0a;
  for (int i = lane; i < slots / per; i += 32) cp_async16(&s->val[buf][per * i], gval + per * i);
  cp_async_commit();
  const int32_t base = static_cast<int32_t>(static_cast<int64_t>(E0) - e0a);
  if (lane <= n) s->rp[buf][lane] = pa - E0 + base;
  if (32 + lane <= n) s->rp[buf][32 + lane] = pb - E0 + base;
  if (lane == 0) {
    s->e0a[buf] = e0a;
    s->r[buf] = r;
    s->n[buf] = n;
    s->lim[buf] = lim;
  }
  return n;
}

// Multiplies the rows of chunk buffer `buf` and writes their Y pieces: lane
// `sub` of group `grp` (G lanes per group, GPW = 32 / G groups per warp).
template <typename VT>
__device__ __forceinline__ void rows_chunk(const RowsStage<VT>* s, int buf, const RowsOperand& p, int G, int GPW,
                                           int grp, int sub) {
  using T = RowsT<VT>;
  using V = typename T::V;
  using AT = typename T::AT;
  constexpr int VC = T::VC;
  V* Y = static_cast<V*>(p.Y);
  const int32_t ldx_bytes = static_cast<int32_t>(p.ldx * static_cast<int64_t>(sizeof(AT)));  // < 2^31 (checked)
  const int64_t ldyv = p.ldy / VC;
  const int kv = (p.k + VC - 1) / VC;
  const int32_t* scol = s->col[buf];
  const VT* sval = s->val[buf];
  const int64_t e0a = s->e0a[buf];
  const int32_t r0 = s->r[buf], n = s->n[buf], lim = s->lim[buf];
  const int32_t* gcol = p.col + e0a;
  const VT* gval = static_cast<const VT*>(p.val) + e0a;
  for (int j = grp; j < n; j += GPW) {
    const int32_t t0 = s->rp[buf][j], t1 = s->rp[buf][j + 1];
    const int64_t yr = p.yperm ? static_cast<int64_t>(__ldg(p.yperm + r0 + j)) : static_cast<int64_t>(r0 + j);
    const int32_t ts = min(t1, lim);  // staged entries of the row end here
    // the X rows of the group's next row into L2, one line each (when a row
    // spans several lanes: with one lane per row the prefetches cost more)
    if (p.pf && G > 1 && j + GPW < n) {
      const int32_t u0 = s->rp[buf][j + GPW], u1 = min(s->rp[buf][j + GPW + 1], lim);
      for (int32_t u = u0 + sub; u < u1 && u < u0 + kRowsUnroll * G; u += G)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const char*>(p.X) +
                                                       static_cast<int64_t>(scol[u]) * static_cast<int64_t>(ldx_bytes)));
    }
    for (int c = sub; c < kv; c += G) {
      // X piece c of row COL: xc + COL * ldx_bytes (one wide multiply-add per entry)
      const char* xc = static_cast<const char*>(p.X) + 16 * c;
      V part[kRowsParts];
#pragma unroll
      for (int u = 0; u < kRowsParts; ++u) zero(part[u]);
      for (int32_t t = t0; t < ts; t += kRowsUnroll) {
        AT av[kRowsUnroll];
        V xv[kRowsUnroll];
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) {
          av[u] = AT(0);
          zero(xv[u]);
          if (t + u < ts) {
            av[u] = T::acc(sval[t + u]);
            xv[u] = __ldg(reinterpret_cast<const V*>(xc + static_cast<int64_t>(scol[t + u]) *
                                                              static_cast<int64_t>(ldx_bytes)));
          }
        }
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) fma_vec(part[u % kRowsParts], av[u], xv[u]);
      }
      for (int32_t t = max(t0, ts); t < t1; t += kRowsUnroll) {  // past the staged part of a long row
        AT av[kRowsUnroll];
        V xv[kRowsUnroll];
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) {
          av[u] = AT(0);
          zero(xv[u]);
          if (t + u < t1) {
            av[u] = T::acc(gval[t + u]);
            xv[u] = __ldg(reinterpret_cast<const V*>(xc + static_cast<int64_t>(__ldg(gcol + t + u)) *
                                                              static_cast<int64_t>(ldx_bytes)));
          }
        }
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) fma_vec(part[u % kRowsParts], av[u], xv[u]);
      }
      add_vec(part[0], part[1]);
      add_vec(part[2], part[3]);
      add_vec(part[0], part[2]);
      store_piece(Y + yr * ldyv + c, part[0], p.k - c * VC);
    }
  }
}

// Lane group of a product with k columns: one lane per 16-byte piece of a
// row, at most 8 (more pieces: passes over the row).
template <typename VT>
__host__ __device__ __forceinline__ int rows_group(int k) {
  const int kv = (k + RowsT<VT>::VC - 1) / RowsT<VT>::VC;
  return kv <= 1 ? 1 : (kv <= 2 ? 2 : (kv <= 4 ? 4 : 8));
}

// Rows [r_lo, b) of the product by one warp: chunk c is multiplied while the
// indices of chunk c + 1 load into the other buffer and the row pointers of
// chunk c + 2 into registers.  Warp-uniform; all 32 lanes take part.
template <typename VT>
__device__ __forceinline__ void rows_range(RowsStage<VT>* s, const RowsOperand& p, int32_t r_lo, int32_t b, int G,
                                           int lane) {
  if (r_lo >= b) return;
  const int GPW = 32 / G, sub = lane % G, grp = lane / G;
  int32_t pa, pb;
  load_rp(p.rowptr, r_lo, b, lane, &pa, &pb);
  int buf = 0;
  int32_t r1 = r_lo + stage_chunk<VT>(s, buf, p, r_lo, b, lane, pa, pb);  // start of the next chunk
  if (r1 < b) load_rp(p.rowptr, r1, b, lane, &pa, &pb);
  while (true) {
    cp_async_wait_all();
    __syncwarp();
    int32_t r2 = b;
    if (r1 < b) {
      r2 = r1 + stage_chunk<VT>(s, buf ^ 1, p, r1, b, lane, pa, pb);
      if (r2 < b) load_rp(p.rowptr, r2, b, lane, &pa, &pb);
    }
    rows_chunk<VT>(s, buf, p, G, GPW, grp, sub);
    __syncwarp();
    if (r1 >= b) break;
    r1 = r2;
    buf ^= 1;
  }
}

}  // namespace rows
}  // namespace maxe
