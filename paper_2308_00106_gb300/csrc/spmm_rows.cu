// spmm_rows.cu -- SpMM Y' = A' X' for matrices with short rows (Section 2's CSR
// product, k right-hand sides): one row per group of G lanes, single-matrix
// launch (the per-warp machinery is in spmm_rows.cuh).
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
#include "spmm_rows.cuh"

namespace maxe {
namespace {

using namespace rows;

constexpr int kRowsWarps = 8;
constexpr int kRowsThreads = 32 * kRowsWarps;
constexpr int64_t kPartE = 512;  // entries of a part (a warp's unit of work), about

struct RowsParams {
  RowsOperand op;
  const int32_t* wrow;
  int32_t nW, Q;
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
  load_rp(p.op.rowptr, r1, b1, lane, &pa, &pb);
  int buf = 0;
  r1 += stage_chunk<VT>(s, buf, p.op, r1, b1, lane, pa, pb);
  bool more = next_start(p, &r1, &P1, &b1);  // (r1, b1): the next chunk
  if (more) load_rp(p.op.rowptr, r1, b1, lane, &pa, &pb);
  while (true) {
    cp_async_wait_all();
    __syncwarp();
    int32_t r2 = r1, b2 = b1;
    int64_t P2 = P1;
    bool more2 = false;
    if (more) {  // stage the next chunk and fetch the row pointers of the one after
      r2 += stage_chunk<VT>(s, buf ^ 1, p.op, r1, b1, lane, pa, pb);
      more2 = next_start(p, &r2, &P2, &b2);
      if (more2) load_rp(p.op.rowptr, r2, b2, lane, &pa, &pb);
    }
    rows_chunk<VT>(s, buf, p.op, G, 32 / G, grp, sub);
    __syncwarp();
    if (!more) break;
    r1 = r2;
    b1 = b2;
    P1 = P2;
    more = more2;
    buf ^= 1;
  }
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
  switch (rows_group<VT>(p.op.k)) {
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
  p.op.rowptr = h->rowptr;
  p.op.col = h->col;
  p.op.val = h->val;
  p.op.X = X;
  p.op.Y = Y;
  p.op.yperm = yperm;
  p.op.ldx = ldx;
  p.op.ldy = ldy;
  p.op.k = k;
  p.op.pf = h->spmm_rows_pf;
  p.wrow = h->wrow[0];
  p.nW = h->nW[0];
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
