// spmm_rows.cu -- SpMM Y' = A' X' for matrices with short rows (Section 2's CSR
// product, k right-hand sides): one row per group of G lanes.
//
// Each lane holds VC = 16 bytes of columns of X and Y (4 FP32 / 2 FP64), so a
// group of G lanes covers G * VC columns (more columns: more passes over the
// row).  A group walks its row's entries, loading the column and value (the
// same address for the G lanes: one request), gathering the 16-byte piece of X
// row COL that is its lanes', and accumulating in registers; it writes its
// piece of Y once.  Entries go eight at a time, their X loads issued
// together, each of the eight into its own partial sum (added at the end in a
// fixed order): shorter dependency chains and a rounding error that grows with
// an eighth of the row's length.
// Warps take the handle's nnz-balanced row ranges, each cut into Q equal
// parts (more warps in flight than the CSR kernel's partition holds); a warp's
// 32 / G groups take rows of its part in turn.  Rows are never split, so each
// Y row is one group's sum in entry order: deterministic, but a long row holds
// its group (and its warp) -- the autotuner keeps this path only for matrices
// where it is faster.  Requires 16-byte aligned X and Y with ldx and ldy
// multiples of VC.
#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kRowsThreads = 256;
constexpr int kRowsUnroll = 8;  // entries per step of a group, each with its own partial sum

template <typename VT>
struct RowsT;
template <>
struct RowsT<float> {
  using AT = float;
  using V = float4;
  static constexpr int VC = 4;
  static __device__ __forceinline__ float val(const void* v, int64_t e) { return __ldg(static_cast<const float*>(v) + e); }
};
template <>
struct RowsT<uint16_t> {
  using AT = float;
  using V = float4;
  static constexpr int VC = 4;
  static __device__ __forceinline__ float val(const void* v, int64_t e) {
    return __uint_as_float(static_cast<uint32_t>(__ldg(static_cast<const unsigned short*>(v) + e)) << 16);
  }
};
template <>
struct RowsT<double> {
  using AT = double;
  using V = double2;
  static constexpr int VC = 2;
  static __device__ __forceinline__ double val(const void* v, int64_t e) {
    return __ldg(static_cast<const double*>(v) + e);
  }
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
__device__ __forceinline__ void zero(float4& v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero(double2& v) { v = make_double2(0.0, 0.0); }

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
};

template <typename VT, int G>
__global__ void __launch_bounds__(kRowsThreads) spmm_rows_kernel(const RowsParams p) {
  using T = RowsT<VT>;
  using V = typename T::V;
  using AT = typename T::AT;
  constexpr int VC = T::VC;
  constexpr int GPW = 32 / G;  // groups per warp
  const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * kRowsThreads + threadIdx.x) >> 5;
  if (gw >= static_cast<int64_t>(p.nW) * p.Q) return;
  const int32_t w = static_cast<int32_t>(gw / p.Q), q = static_cast<int32_t>(gw % p.Q);
  const int32_t a = p.wrow[w], b = p.wrow[w + 1];
  const int64_t len = b - a;
  const int32_t r_lo = a + static_cast<int32_t>(len * q / p.Q), r_hi = a + static_cast<int32_t>(len * (q + 1) / p.Q);
  const V* X = static_cast<const V*>(p.X);
  V* Y = static_cast<V*>(p.Y);
  const int64_t ldxv = p.ldx / VC, ldyv = p.ldy / VC;
  const int kv = (p.k + VC - 1) / VC;  // 16-byte pieces of a row
  for (int32_t r = r_lo + grp; r < r_hi; r += GPW) {
    const int32_t e0 = __ldg(p.rowptr + r), e1 = __ldg(p.rowptr + r + 1);
    const int64_t yr = p.yperm ? static_cast<int64_t>(p.yperm[r]) : static_cast<int64_t>(r);
    for (int c = sub; c < kv; c += G) {
      V part[kRowsUnroll];
#pragma unroll
      for (int u = 0; u < kRowsUnroll; ++u) zero(part[u]);
      int32_t e = e0;
      for (; e + kRowsUnroll <= e1; e += kRowsUnroll) {
        int32_t cj[kRowsUnroll];
        AT av[kRowsUnroll];
        V xv[kRowsUnroll];
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) {
          cj[u] = __ldg(p.col + e + u);
          av[u] = T::val(p.val, e + u);
        }
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) xv[u] = __ldg(X + static_cast<int64_t>(cj[u]) * ldxv + c);
#pragma unroll
        for (int u = 0; u < kRowsUnroll; ++u) fma_vec(part[u], av[u], xv[u]);
      }
#pragma unroll
      for (int u = 0; u < kRowsUnroll - 1; ++u)  // the rest (fewer than eight entries)
        if (e + u < e1)
          fma_vec(part[u], T::val(p.val, e + u), __ldg(X + static_cast<int64_t>(__ldg(p.col + e + u)) * ldxv + c));
      V acc = part[0];
#pragma unroll
      for (int u = 1; u < kRowsUnroll; ++u) add_vec(acc, part[u]);
      if ((c + 1) * VC <= p.k) {
        Y[yr * ldyv + c] = acc;
      } else {  // the row's last, partial piece: only the k columns are written
        AT* y = reinterpret_cast<AT*>(Y + yr * ldyv + c);
        const AT* s = reinterpret_cast<const AT*>(&acc);
        for (int i = 0; i < p.k - c * VC; ++i) y[i] = s[i];
      }
    }
  }
}

template <typename VT>
constexpr int rows_vc() {
  return RowsT<VT>::VC;
}

template <typename VT>
int rows_group(int k) {
  const int kv = (k + rows_vc<VT>() - 1) / rows_vc<VT>();
  return kv <= 1 ? 1 : (kv <= 2 ? 2 : (kv <= 4 ? 4 : 8));
}

template <typename VT>
maxe_status launch_rows(const RowsParams& p, cudaStream_t st) {
  const int g = rows_group<VT>(p.k);
  const int64_t threads = static_cast<int64_t>(p.nW) * p.Q * 32;
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, ceil_div(threads, kRowsThreads)));
  switch (g) {
    case 1: spmm_rows_kernel<VT, 1><<<grid, kRowsThreads, 0, st>>>(p); break;
    case 2: spmm_rows_kernel<VT, 2><<<grid, kRowsThreads, 0, st>>>(p); break;
    case 4: spmm_rows_kernel<VT, 4><<<grid, kRowsThreads, 0, st>>>(p); break;
    default: spmm_rows_kernel<VT, 8><<<grid, kRowsThreads, 0, st>>>(p); break;
  }
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace

bool spmm_rows_ready(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, const void* Y, int64_t ldy) {
  const int vc = h->dtype == MAXE_F64 ? 2 : 4;
  return k >= 1 && ldx % vc == 0 && ldy % vc == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0 &&
         (reinterpret_cast<uintptr_t>(Y) & 15u) == 0;
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
  p.Q = 3;
  switch (h->dtype) {
    case MAXE_F64: return launch_rows<double>(p, st);
    case MAXE_F32: return launch_rows<float>(p, st);
    case MAXE_BF16: return launch_rows<uint16_t>(p, st);
  }
  return MAXE_ERR_INVALID;
}

}  // namespace maxe
