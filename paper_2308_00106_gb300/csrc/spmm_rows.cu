// spmm_rows.cu -- SpMM Y' = A' X' for matrices with short rows (Section 2's CSR
// product, k right-hand sides): one row per group of G lanes.
//
// Each lane holds VC = 16 bytes of columns of X and Y (4 FP32 / 2 FP64), so a
// group of G lanes covers G * VC columns (more columns: more passes over the
// row).  A group walks its row's entries, gathers the 16-byte piece of X row
// COL that is its lanes', accumulates in registers and writes its piece of Y
// once.
//
// The row's column indices come from shared memory, so that the gathers of X
// (the bytes that matter) are the only global loads a row waits for.  A warp
// works through its rows in chunks (at most kChunkR rows and kChunkE entries):
// while it multiplies chunk c, the column indices and values of chunk c + 1
// are on their way into the other half of its double buffer (16-byte cp.async
// copies, rounded out to 8-entry boundaries; the CSR arrays are padded past
// nnz) and the row pointers of chunk c + 2 into registers.  A row longer than
// kChunkE is a chunk of its own; its entries past the staged ones are read
// from global memory.
//
// Entries go eight at a time, their X loads issued together, into four
// partial sums (entries u and u + 4 of a step share one) added in a fixed
// order at the end: shorter dependency chains and a rounding error that grows
// with a quarter of the row's length.  The work is cut into parts of about
// kPartE entries (the handle's nnz-balanced row ranges, each split into Q
// parts of equal row counts); one resident wave of persistent warps takes them
// in turn (warp g: parts g, g + NG, ...), its chunk pipeline running on from
// part to part.  Neighbouring warps hold neighbouring parts, so the rows in
// flight at any time form one window of the matrix and the X rows that nearby
// rows share (a stencil's) are still in L2 when the second one needs them.
// Rows are never split, so each Y row is one group's sum in entry order:
// deterministic, but a long row holds its group (and its warp) -- the autotuner
// keeps this path only for matrices where it is faster.  Requires 16-byte
// aligned X, Y, column and value arrays, with ldx and ldy multiples of VC and
// ldx rows under 2 GiB.
#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kRowsWarps = 8;
constexpr int kRowsThreads = 32 * kRowsWarps;
constexpr int kRowsUnroll = 8;  // entries per step of a group
constexpr int kRowsParts = 4;   // partial sums of a group
constexpr int kChunkE = 256;    // entries of a chunk (a longer row: the first kChunkE)
constexpr int kChunkR = 63;     // rows of a chunk: its 64 row pointers are two per lane
constexpr int kSlotE = kChunkE + 8;  // staged slots: the chunk rounded out to 8-entry boundaries
constexpr int64_t kPartE = 512;  // entries of a part (a warp's unit of work), about

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

struct RowsParams {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  const void* X;
  void* Y;
  const int32_t* yperm;
  const int32_t* wrow;
  int64_t ldx, ldy;
  int32_t k, nW, Q;
  int64_t NG;  // warps of the grid: warp g takes parts g, g + NG, g + 2 NG, ...
};

// Rows [*lo, *hi) of part P: range P / Q of the warp partition, cut into Q
// parts of equal row counts.
__device__ __forceinline__ void part_rows(const RowsParams& p, int64_t P, int32_t* lo, int32_t* hi) {
  const int32_t w = static_cast<int32_t>(P / p.Q), q = static_cast<int32_t>(P % p.Q);
  const int32_t a = __ldg(p.wrow + w), bw = __ldg(p.wrow + w + 1);
  const int64_t len = bw - a;
  *lo = a + static_cast<int32_t>(len * q / p.Q);
  *hi = a + static_cast<int32_t>(len * (q + 1) / p.Q);
}

// The first chunk start at or after row r of part *P (rows up to *b): row r
// itself while r < *b, else the first row of the warp's next non-empty part.
// False when the warp has no parts left.
__device__ __forceinline__ bool next_start(const RowsParams& p, int32_t* r, int64_t* P, int32_t* b) {
  const int64_t NP = static_cast<int64_t>(p.nW) * p.Q;
  while (*r >= *b) {
    *P += p.NG;
    if (*P >= NP) return false;
    part_rows(p, *P, r, b);
  }
  return true;
}

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
__device__ __forceinline__ int32_t stage_chunk(RowsStage<VT>* s, int buf, const RowsParams& p, int32_t r, int32_t b,
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

// Multiplies the rows of chunk buffer `buf` and writes their Y pieces.
template <typename VT, int G>
__device__ __forceinline__ void rows_chunk(const RowsStage<VT>* s, int buf, const RowsParams& p, int grp, int sub) {
  using T = RowsT<VT>;
  using V = typename T::V;
  using AT = typename T::AT;
  constexpr int VC = T::VC;
  constexpr int GPW = 32 / G;
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

template <typename VT, int G>
__global__ void __launch_bounds__(kRowsThreads) spmm_rows_kernel(const RowsParams p) {
  extern __shared__ __align__(16) unsigned char rows_smem[];
  const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
  RowsStage<VT>* s = reinterpret_cast<RowsStage<VT>*>(rows_smem) + (threadIdx.x >> 5);
  // The warp's chunks, part after part, as one sequence: chunk i is multiplied
  // while the indices of chunk i + 1 load into the other buffer and the row
  // pointers of chunk i + 2 into registers.  Neighbouring warps take
  // neighbouring parts, so the rows in flight form one window of the matrix.
  int64_t P1 = (static_cast<int64_t>(blockIdx.x) * kRowsThreads + threadIdx.x) >> 5;
  if (P1 >= static_cast<int64_t>(p.nW) * p.Q) return;
  int32_t r1, b1;
  part_rows(p, P1, &r1, &b1);
  if (!next_start(p, &r1, &P1, &b1)) return;  // steps past an empty first part
  int32_t pa, pb;
  load_rp(p.rowptr, r1, b1, lane, &pa, &pb);
  int buf = 0;
  r1 += stage_chunk<VT>(s, buf, p, r1, b1, lane, pa, pb);
  bool more = next_start(p, &r1, &P1, &b1);  // (r1, b1): the next chunk
  if (more) load_rp(p.rowptr, r1, b1, lane, &pa, &pb);
  while (true) {
    cp_async_wait_all();
    __syncwarp();
    int32_t r2 = r1, b2 = b1;
    int64_t P2 = P1;
    bool more2 = false;
    if (more) {  // stage the next chunk and fetch the row pointers of the one after
      r2 += stage_chunk<VT>(s, buf ^ 1, p, r1, b1, lane, pa, pb);
      more2 = next_start(p, &r2, &P2, &b2);
      if (more2) load_rp(p.rowptr, r2, b2, lane, &pa, &pb);
    }
    rows_chunk<VT, G>(s, buf, p, grp, sub);
    __syncwarp();
    if (!more) break;
    r1 = r2;
    b1 = b2;
    P1 = P2;
    more = more2;
    buf ^= 1;
  }
}

template <typename VT>
constexpr int rows_vc() {
  return RowsT<VT>::VC;
}

// lanes of a row group: one per 16-byte piece of the row, at most 8
template <typename VT>
int rows_group(int k) {
  const int kv = (k + rows_vc<VT>() - 1) / rows_vc<VT>();
  return kv <= 1 ? 1 : (kv <= 2 ? 2 : (kv <= 4 ? 4 : 8));
}

template <typename VT, int G>
maxe_status launch_rows_g(RowsParams p, int sms, cudaStream_t st) {
  static PerDeviceOnce once;
  static int blocks_per_sm[64];
  constexpr size_t smem = sizeof(RowsStage<VT>) * kRowsWarps;
  int dev = 0;
  MAXE_CUDA_TRY(cudaGetDevice(&dev));
  MAXE_TRY(once.run([dev] {
    MAXE_CUDA_TRY(cudaFuncSetAttribute(spmm_rows_kernel<VT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
    int b = 0;
    MAXE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, spmm_rows_kernel<VT, G>, kRowsThreads, smem));
    blocks_per_sm[dev] = std::max(b, 1);
    return MAXE_OK;
  }));
  // one resident wave of persistent warps
  const int64_t parts = static_cast<int64_t>(p.nW) * p.Q;
  p.NG = std::max<int64_t>(1, std::min<int64_t>(parts, static_cast<int64_t>(sms) * blocks_per_sm[dev] * kRowsWarps));
  const unsigned grid = static_cast<unsigned>(ceil_div(p.NG, kRowsWarps));
  spmm_rows_kernel<VT, G><<<grid, kRowsThreads, smem, st>>>(p);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status launch_rows(const RowsParams& p, int sms, cudaStream_t st) {
  switch (rows_group<VT>(p.k)) {
    case 1: return launch_rows_g<VT, 1>(p, sms, st);
    case 2: return launch_rows_g<VT, 2>(p, sms, st);
    case 4: return launch_rows_g<VT, 4>(p, sms, st);
    default: return launch_rows_g<VT, 8>(p, sms, st);
  }
}

}  // namespace

bool spmm_rows_ready(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, const void* Y, int64_t ldy) {
  const int vc = h->dtype == MAXE_F64 ? 2 : 4;
  auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  const int64_t eb = h->dtype == MAXE_F64 ? 8 : 4;
  return k >= 1 && ldx % vc == 0 && ldy % vc == 0 && ldx * eb < (int64_t(1) << 31) && a16(X) && a16(Y) &&
         a16(h->col) && a16(h->val);
}

maxe_status spmm_rows_launch(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                             const int32_t* yperm, cudaStream_t st) {
  if (h->rows == 0 || k == 0) return MAXE_OK;
  RowsParams p{};
  p.rowptr = h->rowptr;
  p.col = h->col;
  p.val = h->val;
  p.X = X;
  p.Y = Y;
  p.yperm = yperm;
  p.wrow = h->wrow[0];
  p.nW = h->nW[0];
  p.ldx = ldx;
  p.ldy = ldy;
  p.k = k;
  // parts of about kPartE entries: a warp's range cut into Q parts of equal row counts
  const int64_t per_range = ceil_div(std::max<int64_t>(h->nnz, 1), std::max(p.nW, 1));
  p.Q = static_cast<int32_t>(std::max<int64_t>(1, ceil_div(per_range, kPartE)));
  const int sms = std::max(h->sms, 1);
  switch (h->dtype) {
    case MAXE_F64: return launch_rows<double>(p, sms, st);
    case MAXE_F32: return launch_rows<float>(p, sms, st);
    case MAXE_BF16: return launch_rows<uint16_t>(p, sms, st);
  }
  return MAXE_ERR_INVALID;
}

}  // namespace maxe
