// spmv.cu -- nnz-balanced CSR SpMV / SpMM on the permuted matrix (Section 2:
// y_i = sum_{l in ROW[i]:ROW[i+1]} V[l] * x[COL[l]];  Eq. 1 for the permuted form).
//
// Work partition (built once per handle).  The nonzeros are cut into nW ranges
// of H entries; warp w owns the rows that START in [w*H, (w+1)*H) (wrow[w] =
// first row with rowptr[r] >= w*H) and streams all of their entries, so every
// warp does H entries give or take one row, whatever the row-length law, and
// no partial sum ever crosses between warps: the load balance the paper's
// laggard argument (Section 1) asks of the permutation, obtained without it.
// nW is the number of warps the GPU keeps resident, so one launch is one wave.
//
// Per warp, the entries go by in pieces of 256 (8 consecutive entries per lane):
//   * COL and VAL of each piece land in the warp's own shared-memory ring by
//     1-D bulk copies (TMA, L2 evict-first: the matrix is read once per
//     product), kStages pieces ahead, completion on one mbarrier per stage, so
//     prefetching costs no registers;
//   * the row pointers of the rows that end in the piece (32 per load, one
//     piece ahead) mark the row starts in a 256-bit shared-memory bitmap;
//   * x[COL] is gathered through L1/L2 and multiplied in registers;
//   * a segmented inclusive scan (serial over the lane's 8 entries, 5 shuffle
//     steps across lanes) sums each row; the partial row that runs on into the
//     next piece is kept as the warp's carry;
//   * each row that ends in the piece reads its sum back from the scan and is
//     written once, optionally through rperm (y = P_r^{-1} y' fused into the
//     epilogue).
// The result depends only on the matrix and the partition: deterministic.
//
// SpMM: X rows are gathered VW columns at a time (float4 / float2 / double2),
// and the scan runs on VW-wide vectors, one pass per group of VW columns.
#include <algorithm>

#include "spmv_warp.cuh"

namespace maxe {
namespace {

using namespace warp;

template <typename VT, int VW, int IT, bool UNIT>
maxe_status prepare_variant() {
  static PerDeviceOnce once;  // the attribute is per function and device
  return once.run([] {
    MAXE_CUDA_TRY(cudaFuncSetAttribute(spmm_warp_kernel<Cfg<VT, VW, IT, UNIT>>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(block_smem<VT, VW, IT>())));
    return MAXE_OK;
  });
}

template <typename VT, int VW, int IT, bool UNIT>
maxe_status launch_variant(const Params& p, cudaStream_t st) {
  MAXE_TRY((prepare_variant<VT, VW, IT, UNIT>()));
  const unsigned grid = static_cast<unsigned>(ceil_div(p.nW, kWarps));
  spmm_warp_kernel<Cfg<VT, VW, IT, UNIT>><<<grid, kThreads, block_smem<VT, VW, IT>(), st>>>(p);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status launch_lc(const Params& p, int g, cudaStream_t st) {
  static PerDeviceOnce once;
  const size_t smem = sizeof(WarpSmemLC<VT>) * kWarps;
  MAXE_TRY(once.run([smem] {
    MAXE_CUDA_TRY(cudaFuncSetAttribute(spmm_lc_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem)));
    return MAXE_OK;
  }));
  const unsigned grid = static_cast<unsigned>(ceil_div(p.nW, kWarps));
  spmm_lc_kernel<VT><<<grid, kThreads, smem, st>>>(p, g);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

// it: 0 -> 8 entries per lane, 1 -> 16 (SpMV with unit strides only)
template <typename VT>
maxe_status launch_dtype(const Params& p, int vw, int it, bool unit, cudaStream_t st) {
  if (vw == 1) {
    if (unit) return it ? launch_variant<VT, 1, 16, true>(p, st) : launch_variant<VT, 1, 8, true>(p, st);
    return launch_variant<VT, 1, 8, false>(p, st);
  }
  if (vw == 2) return launch_variant<VT, 2, 8, false>(p, st);
  if constexpr (sizeof(typename Acc<VT>::T) == 4) {
    if (vw == 4) return launch_variant<VT, 4, 8, false>(p, st);
  }
  return MAXE_ERR_UNSUPPORTED;
}

template <typename VT, int IT>
int resident_warps(int sms) {
  int blocks = 0;
  if (prepare_variant<VT, 1, IT, true>() != MAXE_OK ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, spmm_warp_kernel<Cfg<VT, 1, IT, true>>, kThreads,
                                                    block_smem<VT, 1, IT>()) != cudaSuccess ||
      blocks < 1) {
    cudaGetLastError();
    blocks = 1;
  }
  return sms * blocks * kWarps;
}

template <int IT>
int resident_for(maxe_dtype d, int sms) {
  switch (d) {
    case MAXE_F64: return resident_warps<double, IT>(sms);
    case MAXE_F32: return resident_warps<float, IT>(sms);
    case MAXE_BF16: return resident_warps<uint16_t, IT>(sms);
  }
  return sms * kWarps;
}

}  // namespace

int64_t spmv_pad_elems() { return 32 * kMaxItems * kStages + 8; }

namespace {

// wrow[w] = w * M / nW: the same number of rows for every warp, whatever they hold.
__global__ void equal_rows_kernel(int32_t* __restrict__ wrow, int64_t nW, int64_t M) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w <= nW) wrow[w] = static_cast<int32_t>(w * M / nW);
}

}  // namespace

maxe_status spmv_build_partition(maxe_handle* h, cudaStream_t st) {
  for (int v = 0; v < 2; ++v) {
    const int target = v == 0 ? resident_for<8>(h->dtype, h->sms) : resident_for<16>(h->dtype, h->sms);
    if (h->equal_rows) {
      const int64_t nW = std::max<int64_t>(1, std::min<int64_t>(target, h->rows));
      h->wrow[v] = static_cast<int32_t*>(h->al.get(static_cast<size_t>(nW + 1) * sizeof(int32_t)));
      if (!h->wrow[v]) return MAXE_ERR_OOM;
      h->nW[v] = static_cast<int32_t>(nW);
      equal_rows_kernel<<<static_cast<unsigned>(ceil_div(nW + 1, 256)), 256, 0, st>>>(h->wrow[v], nW, h->rows);
      MAXE_CUDA_TRY(cudaGetLastError());
      continue;
    }
    const int64_t H = std::max<int64_t>(256, ceil_div(std::max<int64_t>(h->nnz, 1), std::max(target, 1)));
    const int64_t nW = std::max<int64_t>(1, ceil_div(h->nnz, H));
    h->wrow[v] = static_cast<int32_t*>(h->al.get(static_cast<size_t>(nW + 1) * sizeof(int32_t)));
    if (!h->wrow[v]) return MAXE_ERR_OOM;
    h->nW[v] = static_cast<int32_t>(nW);
    // wrow[w] = min{ r : rowptr[r] >= w*H }; the last range also takes trailing empty rows
    MAXE_TRY(bucket_lower_bounds(h->rowptr, h->rows, H, 0, nW, h->wrow[v], st));
    MAXE_TRY(set_i32(h->wrow[v] + nW, h->rows, st));
  }
  return MAXE_OK;
}

maxe_status spmm_launch(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        const int32_t* yperm, cudaStream_t st, int variant, int lc) {
  if (h->rows == 0 || k == 0) return MAXE_OK;
  if (h->nnz == 0) {  // Y = 0 whatever X holds; X is not read (with no columns it holds nothing)
    const size_t eb = static_cast<size_t>(vector_bytes(h->dtype));
    MAXE_CUDA_TRY(cudaMemset2DAsync(Y, static_cast<size_t>(ldy) * eb, 0, static_cast<size_t>(k) * eb,
                                    static_cast<size_t>(h->rows), st));
    return MAXE_OK;
  }
  Params p{};
  p.rowptr = h->rowptr;
  p.col = h->col;
  p.val = h->val;
  p.X = X;
  p.Y = Y;
  p.yperm = yperm;
  p.status = h->status;
  p.wait_ns = wait_limit_ns(h->device);
  p.ldx = ldx;
  p.ldy = ldy;
  p.k = k;
  p.M = h->rows;
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
  const bool unit = k == 1 && ldx == 1 && ldy == 1;
  if (unit && variant < 0 && lc < 0 && xslice_ready(h, X)) return xslice_launch(h, X, Y, yperm, st);
  if (k > 1 && variant < 0 && lc < 0 && h->spmm_rows && spmm_rows_ready(h, k, X, ldx, Y, ldy))
    return spmm_rows_launch(h, k, X, ldx, Y, ldy, yperm, st);
  const int it = (unit && variant < 0) ? h->spmv_items16 : (variant > 0 ? 1 : 0);
  if (it == 1 && !unit) return MAXE_ERR_UNSUPPORTED;
  p.wrow = h->wrow[it];
  p.nW = h->nW[it];
  // k columns across lanes when the rows of X and Y hold whole vectors
  const int g = lc_group(k, eb, static_cast<int>(ldx % 1024), static_cast<int>(ldy % 1024));
  const bool use_lc = lc < 0 ? h->spmm_lc != 0 : lc != 0;
  if (g > 0 && use_lc && aligned(eb == 4 ? 4 : 2)) {
    switch (h->dtype) {
      case MAXE_F64: return launch_lc<double>(p, g, st);
      case MAXE_F32: return launch_lc<float>(p, g, st);
      case MAXE_BF16: return launch_lc<uint16_t>(p, g, st);
    }
  }
  switch (h->dtype) {
    case MAXE_F64: return launch_dtype<double>(p, vw, it, unit, st);
    case MAXE_F32: return launch_dtype<float>(p, vw, it, unit, st);
    case MAXE_BF16: return launch_dtype<uint16_t>(p, vw, it, unit, st);
  }
  return MAXE_ERR_INVALID;
}

maxe_status spmv_autotune(maxe_handle* h, cudaStream_t st) {
  if (h->rows == 0 || h->nnz == 0) return MAXE_OK;
  ScratchSet scratch(h->al);
  const int eb = vector_bytes(h->dtype);
  void* x = scratch.get<unsigned char>(static_cast<size_t>(h->cols) * eb);
  void* y = scratch.get<unsigned char>(static_cast<size_t>(h->rows) * eb);
  if (!x || !y) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemsetAsync(x, 0, static_cast<size_t>(h->cols) * eb, st));
  cudaEvent_t e0, e1;
  MAXE_CUDA_TRY(cudaEventCreate(&e0));
  MAXE_CUDA_TRY(cudaEventCreate(&e1));
  // time(launch) over 5 launches after 2 warm-up launches
  auto timed = [&](auto&& launch, float* ms) -> maxe_status {
    maxe_status s = MAXE_OK;
    for (int rep = 0; rep < 2 && s == MAXE_OK; ++rep) s = launch();
    if (s != MAXE_OK) return s;
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 5 && s == MAXE_OK; ++rep) s = launch();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return MAXE_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return s;
  };
  float best = 1e30f;
  int pick = 0;
  maxe_status s = MAXE_OK;
  for (int v = 0; v < 2 && s == MAXE_OK; ++v) {
    float ms = 0.f;
    s = timed([&] { return spmm_launch(h, 1, x, 1, y, 1, nullptr, st, v); }, &ms);
    if (s == MAXE_OK && ms < best) {
      best = ms;
      pick = v;
    }
  }
  h->spmv_items16 = pick;
  // the x-sliced kernel, when the handle has it
  if (s == MAXE_OK && h->xs_idx) {
    // and its stream prefetch distance (entries; 0: none)
    const int32_t dist[4] = {0, 512, 1024, 2048};
    float best_xs = 1e30f;
    int32_t pick_d = 0;
    for (int d = 0; d < 4 && s == MAXE_OK; ++d) {
      h->xs_ahead = dist[d];
      float ms = 0.f;
      s = timed([&] { return xslice_launch(h, x, y, nullptr, st); }, &ms);
      if (s == MAXE_OK && ms < best_xs) {
        best_xs = ms;
        pick_d = dist[d];
      }
    }
    h->xs_ahead = pick_d;
    if (s == MAXE_OK) h->xs_use = best_xs < best ? 1 : 0;
  }
  // SpMM path for wide right-hand sides, timed at k = 16 when the scratch is modest
  const int64_t k = 16;
  const int64_t bytes = (static_cast<int64_t>(h->rows) + h->cols) * k * eb;
  if (s == MAXE_OK && bytes <= (int64_t(8) << 30)) {
    void* X = h->al.get(static_cast<size_t>(h->cols) * k * eb);
    void* Y = h->al.get(static_cast<size_t>(h->rows) * k * eb);
    if (X && Y) {
      s = cudaMemsetAsync(X, 0, static_cast<size_t>(h->cols) * k * eb, st) == cudaSuccess ? MAXE_OK : MAXE_ERR_CUDA;
      float t_pass = 0.f, t_lc = 0.f, t_rows = 0.f;
      if (s == MAXE_OK) s = timed([&] { return spmm_launch(h, k, X, k, Y, k, nullptr, st, -1, 0); }, &t_pass);
      if (s == MAXE_OK) s = timed([&] { return spmm_launch(h, k, X, k, Y, k, nullptr, st, -1, 1); }, &t_lc);
      const bool rows_ok = spmm_rows_ready(h, static_cast<int32_t>(k), X, k, Y, k);
      if (s == MAXE_OK && rows_ok) {  // with and without its next-row prefetch
        float t_pf = 0.f;
        h->spmm_rows_pf = 0;
        s = timed([&] { return spmm_rows_launch(h, k, X, k, Y, k, nullptr, st); }, &t_rows);
        h->spmm_rows_pf = 1;
        if (s == MAXE_OK) s = timed([&] { return spmm_rows_launch(h, k, X, k, Y, k, nullptr, st); }, &t_pf);
        h->spmm_rows_pf = t_pf < t_rows ? 1 : 0;
        t_rows = std::min(t_rows, t_pf);
      }
      if (s == MAXE_OK) {
        h->spmm_lc = t_lc < t_pass ? 1 : 0;
        h->spmm_rows = rows_ok && t_rows < std::min(t_pass, t_lc) ? 1 : 0;
      }
    }
    h->al.put(Y);
    h->al.put(X);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // namespace maxe
