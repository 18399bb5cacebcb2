// handle.cuh -- layout of the library-owned permuted matrix (not part of the ABI).
//
// HBM layout of a handle (all int32 indices):
//   rowptr  [rows + 1 + kRowptrPad]        row pointers of A' = P_r A P_c
//   col     [nnz_pad]                      columns, ascending per row, zero padded
//   val     [nnz_pad]                      values (f64 / f32 / bf16 bits), zero padded
//   wrow    [nW + 1]                       SpMV work partition: first row of each warp range
//   rperm, cperm [rows], [cols]            copies of the permutations (or NULL)
//   xbuf                                   x' = P_c^{-1} x scratch for original-space calls
//   coo_row [nnz], coo_carry               COO form (MAXE_COO): row of each entry, and
//                                          per-256-entry-chunk partial sums + flags
// nnz_pad leaves at least two 128-entry pieces of zeros after the last entry,
// so the SpMV warps can load whole aligned pieces (and prefetch one ahead)
// without a bounds test.
#pragma once

#include "internal.cuh"

struct maxe_handle {
  int32_t rows = 0, cols = 0;
  int64_t nnz = 0, nnz_pad = 0;
  maxe_dtype dtype = MAXE_F32;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  void* val = nullptr;
  int32_t* rperm = nullptr;
  int32_t* cperm = nullptr;
  int32_t* wrow[2] = {nullptr, nullptr};  // per SpMV variant (8 / 16 entries per lane)
  int32_t nW[2] = {0, 0};
  int spmv_items16 = 0;                    // chosen SpMV variant (autotuned or 0)
  int spmm_lc = 0;                         // SpMM with columns across lanes (autotuned or 0)
  int spmm_rows = 0;                       // SpMM with one row per lane group (autotuned or 0)
  int spmm_rows_pf = 0;                    // that kernel prefetches each group's next X rows (autotuned)
  int equal_rows = 0;                      // SpMV partition: equal rows per warp (not equal nonzeros)
  int32_t* bwrow = nullptr;                // batch plan: partition with bH entries per warp task
  int32_t bnW = 0;
  int64_t bH = 0;
  int bit16 = 0;                           // batch plan: 16 entries per lane for k = 1
  int blc = 0;                             // batch plan, SpMM: 0 column passes, 1 columns across lanes, 2 rows
  int bbps = 0;                            // batch plan: CTAs per SM of its launch (0: as many as fit)
  // x-sliced SpMV form (MAXE_XSLICE): entries grouped by ((tile, half, warp range), column slice)
  uint32_t* xs_idx = nullptr;              // (accumulator << 15) | column in slice, step-major cells;
                                           // with FP32 values (index, value bits) pairs
  void* xs_val = nullptr;                  // BF16 / FP64 values beside xs_idx (null for FP32)
  int32_t* xs_seg = nullptr;               // [3 * cells]: first entry, steps, full lanes | partial entries << 6
  int64_t xs_cells = 0;
  int32_t* xs_tile_row = nullptr;          // [ntiles + 1]
  int32_t* xs_warp_row = nullptr;          // [ntiles * pair * 16], xs_vslot follows in the same block
  int32_t* xs_vslot = nullptr;
  int32_t* xs_vl_off = nullptr;            // [ntiles * pair * 15 + 1], xs_vl_item follows in the same block
  int32_t* xs_vl_item = nullptr;
  int32_t* xs_tl_off = nullptr;            // [ntiles * pair + 1], xs_tl_slice follows in the same block
  int32_t* xs_tl_slice = nullptr;
  int32_t xs_ntiles = 0, xs_nS = 0;
  int32_t xs_pair = 1;                     // column halves per tile: 1, or 2 on a cluster of two CTAs
  int32_t xs_smem = 0;                     // dynamic shared memory per CTA
  int64_t xs_bytes = 0;
  int64_t xs_nent = 0;                     // entries allocated in xs_idx / xs_val (with the zeroed slack)
  int32_t xs_ahead = 0;                    // L2 prefetch distance (entries) of the x-sliced stream, 0: none
  int xs_use = 0;                          // SpMV (k = 1) takes the x-sliced kernel
  int xs_prefetch = 0;                     // cells large enough for the L2 prefetch cursor
  int32_t* coo_row = nullptr;              // COO row index of every entry (MAXE_COO), else NULL
  void* coo_carry = nullptr;               // COO per-chunk partial sums and flags
  void* xbuf = nullptr;  // cols * k_cap vector elements
  int32_t xbuf_k = 0;
  maxe::Allocator al;
  int device = 0;
  int sms = 0;
  unsigned* status = nullptr;
};

namespace maxe {

inline int value_bytes(maxe_dtype d) { return d == MAXE_F64 ? 8 : (d == MAXE_F32 ? 4 : 2); }
inline int vector_bytes(maxe_dtype d) { return d == MAXE_F64 ? 8 : 4; }

// spmv.cu
int64_t spmv_pad_elems();
maxe_status spmv_build_partition(maxe_handle* h, cudaStream_t st);
// Y = A' X (rows of Y optionally scattered through yperm).  X: cols x k (ldx),
// Y: rows x k (ldy), vector element type of the handle.
// variant: -1 = the handle's choice, 0 / 1 = force 8 / 16 entries per lane;
// lc: -1 = the handle's choice, 0 / 1 = force column passes / columns across lanes.
maxe_status spmm_launch(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        const int32_t* yperm, cudaStream_t st, int variant = -1, int lc = -1);
// Time the SpMV variants on this matrix and keep the faster (synchronises).
maxe_status spmv_autotune(maxe_handle* h, cudaStream_t st);

// batch.cu
constexpr int64_t kDefaultBatchTask = 2048;  // entries per warp task of the default batch plan
maxe_status batch_plan(maxe_handle* h, int64_t H, int it16, cudaStream_t st, int lc, int bps = 0);
maxe_status batch_plan_default(maxe_handle* h, cudaStream_t st);

// spmm_rows.cu: Y = A' X with one row per group of lanes (short rows), when X
// and Y are 16-byte aligned with whole 16-byte pieces per row.
bool spmm_rows_ready(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, const void* Y, int64_t ldy);
maxe_status spmm_rows_launch(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                             const int32_t* yperm, cudaStream_t st);

// xslice.cu: build the x-sliced form (unless forced, leaves it unbuilt when it
// would not pay; pairs: > 0 column halves on CTA pairs, 0 when the halves are
// even, < 0 never); launch y' = A' x' with it (x 16-byte aligned, unit
// strides); free it.
maxe_status xslice_build(maxe_handle* h, cudaStream_t st, bool force, int pairs);
bool xslice_ready(const maxe_handle* h, const void* x);
maxe_status xslice_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st);
void xslice_release(maxe_handle* h);

// coo.cu: the COO row indices and chunk carries of a handle; y = A' x over them
// (rows optionally scattered through yperm).
maxe_status coo_build(maxe_handle* h, cudaStream_t st);
maxe_status coo_spmv_launch(const maxe_handle* h, const void* x, void* y, const int32_t* yperm, cudaStream_t st);

// entropy.cu
maxe_status entropy_run(const maxe_handle* h, int32_t gr, int32_t gc, double base, double* H_host,
                        int64_t* counts_dev, const Allocator& al, cudaStream_t st);

// permute_csr.cu
maxe_status permute_csr_run(const maxe_csr* A, const int32_t* rperm, const int32_t* cperm, uint32_t flags,
                            maxe_handle* h, cudaStream_t st);

// power.cu
maxe_status power_iteration_run(const maxe_handle* h, const void* v0, int32_t steps, void* v_out,
                                double* lambda_host, double* hist_host, cudaStream_t st);

}  // namespace maxe
