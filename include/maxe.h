/*
 * maxe.h -- C ABI of libmaxe.so: entropy-maximising random permutation of a
 * sparse matrix and CSR SpMV/SpMM on the permuted matrix, for NVIDIA GB300
 * (sm_103a).  Jain, Bustany, Fraisse, Benipal, Gaitonde, D'Alberto,
 * "Entropy Maximization in Sparse Matrix by Vector Multiplication", arXiv 2308.00106.
 *
 * The method (Section 1, Eq. 1):  (P_r y) = (P_r A P_c) (P_c^{-1} x).
 * Permutation convention used everywhere: perm[new] = old.  Hence
 *   A'[i', j'] = A[rperm[i'], cperm[j']],   x'[j'] = x[cperm[j']],   y[rperm[i']] = y'[i'].
 *
 * Conventions of every entry point
 *   - Pointers marked (device) are CUDA device pointers of the current device;
 *     (host) are ordinary host pointers.  Arrays are dense, contiguous, and
 *     owned by the caller unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every call is stream-ordered and returns without synchronising, except
 *     maxe_nnz_entropy, maxe_power_iteration and maxe_device_status, which
 *     synchronise `stream` because they return a host value.
 *   - Every call returns a maxe_status.  Argument checks run on the host before
 *     any launch; a failing check launches nothing.  Launch errors surface as
 *     MAXE_ERR_CUDA; asynchronous kernel errors surface on the next
 *     synchronising call.  No C++ exception crosses the ABI.
 *   - Index type is int32: rows, cols and nnz must each be <= INT32_MAX - 64.
 *   - Device-side waits are bounded: a wait that runs out records
 *     MAXE_ERR_TIMEOUT, the kernel returns, and maxe_device_status reports it.
 *   - Results are deterministic: the same inputs, seed and handle give the same
 *     bits on every run.
 */
#ifndef MAXE_H
#define MAXE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MAXE_API __attribute__((visibility("default")))
#else
#define MAXE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MAXE_OK = 0,
  MAXE_ERR_INVALID = 1,     /* bad argument (checked on the host, nothing launched) */
  MAXE_ERR_OOM = 2,         /* the allocator returned NULL */
  MAXE_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  MAXE_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
  MAXE_ERR_UNSUPPORTED = 5  /* valid request the library does not implement */
} maxe_status;

/* Stored value type of a matrix.  Vectors are FP64 for MAXE_F64 matrices and
 * FP32 otherwise; accumulation is FP64 for MAXE_F64 and FP32 otherwise. */
typedef enum { MAXE_F64 = 0, MAXE_F32 = 1, MAXE_BF16 = 2 } maxe_dtype;

/* Flags of maxe_spmv / maxe_spmm: x and y are already in the permuted space
 * (x' and y' of Eq. 1), so no vector permutation is done.  This is the
 * iterative use the paper has in mind (the matrix is reused, Section 1). */
#define MAXE_VEC_PERMUTED 0x1u
/* Flag of maxe_permute_csr: check on the device that rowptr is monotone, columns
 * are in range and perms are bijections (synchronises; MAXE_ERR_INVALID on failure). */
#define MAXE_VALIDATE 0x2u
/* Flag of maxe_permute_csr: time the SpMV kernel variants (8 or 16 entries
 * per lane) on this matrix and keep the faster one for the handle, the same
 * for the x-sliced form when the handle has one; also time the three SpMM
 * paths (column passes, columns across lanes, one row per lane group) at
 * k = 16 when their scratch (rows + cols) * 16 vectors fits in 8 GiB, and keep
 * the fastest (synchronises; a few products of device time). */
#define MAXE_AUTOTUNE 0x4u
/* Flag of maxe_permute_csr: use the 16-entries-per-lane SpMV variant without
 * timing (tuning override; MAXE_AUTOTUNE takes precedence). */
#define MAXE_ITEMS16 0x8u
/* Flag of maxe_permute_csr: SpMM with columns across lanes (groups of lanes
 * hold the k columns, each walks consecutive entries) instead of column passes,
 * for k >= 5 (FP32 vectors) / k >= 3 (FP64) with 16-byte rows of X and Y
 * (tuning override; MAXE_AUTOTUNE takes precedence). */
#define MAXE_SPMM_LANES 0x10u
/* Flag of maxe_permute_csr: split the SpMV work into equal numbers of rows
 * per warp instead of equal numbers of nonzeros.  This is the fixed row
 * partition under which the paper finds that random permutation balances the
 * load (Section 6, parallel CSR and GPU CSR by equal rows). */
#define MAXE_EQUAL_ROWS 0x20u
/* Flag of maxe_permute_csr: also keep the COO form of A' (Section 2: triplets
 * ROW, COL, VALUE) -- a row index per entry beside the CSR's columns and
 * values -- for maxe_coo_spmv.  Costs 4 bytes per entry plus 17 bytes (FP64:
 * 17, else 9) per 256 entries. */
#define MAXE_COO 0x40u
/* Flag of maxe_permute_csr: also build the x-sliced form of A' and use it for
 * SpMV (k = 1, 16-byte aligned x).  The columns are cut into slices of x that
 * fit in shared memory (64 KB: 16384 FP32 / 8192 FP64 columns; 48 KB with
 * column halves), the rows into one tile per SM; each tile's warps own row
 * ranges and read their entries slice by slice, gathering x from shared memory
 * instead of L2 (one L2 request per nonzero on a randomly permuted matrix is
 * what bounds the CSR kernel there).  When the nonzeros of every tile split
 * evenly between the two halves of the columns (FP32 and BF16 values), a tile
 * runs on a cluster of two CTAs, one per half, whose sums are added in a fixed
 * order.  Costs 4 + value-size bytes per entry more memory (plus 12 bytes of
 * descriptor per (row range, slice) cell) and a synchronising build.
 * MAXE_AUTOTUNE builds it too when its x traffic would stay under eight times
 * the matrix, and keeps it only if it times faster than the CSR kernel.
 * Ignored with MAXE_EQUAL_ROWS.  Deterministic. */
#define MAXE_XSLICE 0x80u
/* Tuning overrides of the x-sliced form (with MAXE_XSLICE or MAXE_AUTOTUNE):
 * MAXE_XS_PAIRS runs every tile on a cluster of two CTAs, one per half of the
 * columns, even when the halves are uneven (FP32 and BF16 values; FP64 values
 * never use pairs); MAXE_XS_SINGLE never does.  Not both. */
#define MAXE_XS_PAIRS 0x100u
#define MAXE_XS_SINGLE 0x200u
/* Flag of maxe_permute_csr: SpMM (k > 1) with one row per group of lanes --
 * each lane holds 16 bytes of the k columns of X and Y (4 FP32 / 2 FP64), a
 * group walks its row's entries and writes its piece of Y once -- for matrices
 * with short rows, when X and Y are 16-byte aligned and ldx, ldy are multiples
 * of 4 (FP32 vectors) / 2 (FP64) (tuning override; MAXE_AUTOTUNE times it
 * against the other SpMM paths at k = 16 and keeps the fastest). */
#define MAXE_SPMM_ROWS 0x400u
/* Flag of maxe_permute_csr: with MAXE_SPMM_ROWS, each lane group also
 * prefetches into L2 the X rows of its next row while it sums the current one
 * (tuning override; MAXE_AUTOTUNE times the rows kernel with and without it).
 * Results do not depend on it. */
#define MAXE_SPMM_ROWS_PF 0x800u

/* Device memory allocator used for everything a handle owns and for scratch.
 * alloc(bytes, ctx, stream) returns a device pointer aligned to >= 256 bytes or
 * NULL; free(ptr, ctx, stream) releases it.  Passing NULL where a
 * `const maxe_allocator*` is expected selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, void* ctx, void* stream);
  void* ctx;
} maxe_allocator;

/* A CSR matrix (Section 2: arrays V, COL, ROW): row i holds entries
 * rowptr[i] .. rowptr[i+1]-1; col / val hold their columns and values.
 * All pointers are (device), caller-owned, read-only for the library.
 * rowptr has rows+1 entries, rowptr[0] = 0, rowptr[rows] = nnz. */
typedef struct {
  int32_t rows, cols;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  maxe_dtype dtype;
} maxe_csr;

/* Opaque, library-owned permuted matrix: the CSR of A' = P_r A P_c with
 * ascending columns, the permutations, and the work partition of the SpMV
 * kernel.  Owned arrays come from the allocator given at creation. */
typedef struct maxe_handle maxe_handle;

/* a1 + a2.  Random permutation of 0..n-1 (Section 3; seeded per the
 * "Measuring" section's repeated runs).  key(seed, tag, i) is output number
 * 2*i + tag + 1 of SplitMix64 seeded with `seed`; perm lists 0..n-1 in
 * ascending (key, i) order.  tag 0 is used for rows, 1 for columns.
 * perm: (device) int32[n], written.  alloc: scratch allocator (nullable).
 * Errors: INVALID if n < 0, tag not in {0,1}, or perm NULL with n > 0. */
MAXE_API maxe_status maxe_build_permutation(uint64_t seed, int32_t n, int32_t tag, int32_t* perm,
                                   const maxe_allocator* alloc, void* stream);

/* inv[perm[i]] = i (Eq. 1 needs P^{-1}).  perm, inv: (device) int32[n].
 * perm must be a bijection (not checked here; see MAXE_VALIDATE). */
MAXE_API maxe_status maxe_invert_permutation(const int32_t* perm, int32_t n, int32_t* inv, void* stream);

/* f1.  Nonzero histogram along one axis (Section 5 and the appendix's
 * gradient-based permutations): axis 0 writes hist[i] = entries of row i
 * (rows values), axis 1 writes hist[j] = entries of column j (cols values).
 * A: (device arrays) the CSR; only rowptr (axis 0) or col (axis 1) is read.
 * hist: (device) int32, written.  Exact (integer counts); stream-ordered.
 * Errors: INVALID on a NULL pointer that is needed, axis not in {0,1}. */
MAXE_API maxe_status maxe_nnz_histogram(const maxe_csr* A, int32_t axis, int32_t* hist, void* stream);

/* f1.  Gradient-based permutation of n rows or columns (the appendix's
 * "gradient based row permutation"; Section 5, Figures 4-5):
 *   1. g_i = hist[i+1] - hist[i] for i = 0..n-2;
 *   2. the cut is after the first i of maximum |g_i|: part one is [0, pivot),
 *      part two [pivot, n), pivot = i + 1 (pivot = n when n < 2);
 *   3. the parts are riffled, one card from each in turn starting with part
 *      one, the longer part's remainder following in order;
 *   4. each half of the shuffled deck (its first ceil(n/2) positions, and the
 *      rest) is put in random order: the positions q of a half are sorted by
 *      (key(seed, tag, q), q), the key of maxe_build_permutation.
 * perm[new] = old, as for maxe_build_permutation; apply it with
 * maxe_permute_csr (rows: tag 0 and the row histogram; columns: tag 1 and the
 * column histogram).  hist: (device) int32[n] >= 0; perm: (device) int32[n],
 * written; pivot: (device) int32[1] or NULL, receives the cut.  Deterministic.
 * Errors: INVALID if n < 0, tag not in {0,1} or a needed pointer is NULL;
 * OOM from the allocator. */
MAXE_API maxe_status maxe_gradient_permutation(const int32_t* hist, int32_t n, uint64_t seed, int32_t tag,
                                               int32_t* perm, int32_t* pivot, const maxe_allocator* alloc,
                                               void* stream);

/* a5.  Vector permutation of Eq. 1.  gather: out[i] = in[perm[i]] (x' = P_c^{-1} x);
 * scatter: out[perm[i]] = in[i] (y = P_r^{-1} y').  elem_bytes in {2, 4, 8};
 * in, out: (device) arrays of n elements, must not overlap. */
MAXE_API maxe_status maxe_permute_gather(const int32_t* perm, int32_t n, int32_t elem_bytes, const void* in,
                                void* out, void* stream);
MAXE_API maxe_status maxe_permute_scatter(const int32_t* perm, int32_t n, int32_t elem_bytes, const void* in,
                                 void* out, void* stream);

/* a3.  Build the permuted matrix A' = P_r A P_c (Eq. 1) in CSR with ascending
 * columns (Section 2): new row i' is old row rperm[i']; old column c becomes
 * cinv[c]; each row is then sorted by new column (stable).  Values are copied
 * bit for bit.  rperm (rows) / cperm (cols): (device) int32, NULL = identity
 * (the "plain" matrix).  The handle keeps its own copies of the permutations.
 * flags: any of MAXE_VALIDATE, MAXE_AUTOTUNE, MAXE_ITEMS16, MAXE_SPMM_LANES,
 * MAXE_EQUAL_ROWS, MAXE_COO, MAXE_XSLICE, MAXE_XS_PAIRS, MAXE_XS_SINGLE,
 * MAXE_SPMM_ROWS.  *out receives the new handle.
 * Synchronises `stream` once (to size the pass over rows longer than 2048).
 * Errors: INVALID on bad sizes/NULL pointers (or failed validation), OOM. */
MAXE_API maxe_status maxe_permute_csr(const maxe_csr* A, const int32_t* rperm, const int32_t* cperm,
                             uint32_t flags, const maxe_allocator* alloc, void* stream,
                             maxe_handle** out);

/* Borrow the permuted CSR arrays (device pointers owned by the handle, valid
 * until maxe_handle_destroy).  rperm/cperm (nullable outputs) receive the
 * handle's permutation arrays, NULL for identity. */
MAXE_API maxe_status maxe_handle_csr(const maxe_handle* h, maxe_csr* view_out, const int32_t** rperm,
                            const int32_t** cperm);

/* Kernel variants of the handle, as chosen by MAXE_AUTOTUNE / MAXE_ITEMS16 /
 * MAXE_SPMM_LANES at creation: *items = entries per lane of the SpMV variant
 * (8 or 16), plus 0x100 when SpMM uses columns across lanes, plus 0x200 when
 * SpMV uses the x-sliced form (MAXE_XSLICE), plus 0x400 when that form's cells
 * are large enough for its L2 prefetch cursor, plus 0x800 when it runs its tiles
 * on pairs of CTAs (column halves), plus 0x1000 when SpMM takes one row per
 * group of lanes (MAXE_SPMM_ROWS), plus the SpMM kernel of the batch plan in
 * bits 13-14 (0 column passes, 1 columns across lanes, 2 one row per lane
 * group), plus in bits 15-17 the x-sliced form's L2 prefetch distance along
 * its entry stream in units of 512 entries (0: none; picked by MAXE_AUTOTUNE),
 * plus 0x40000 when the one-row-per-lane-group SpMM prefetches each lane
 * group's next X rows into L2 (picked by MAXE_AUTOTUNE: it pays where
 * neighbouring rows share X rows, as in a stencil, and costs on permuted
 * matrices).  items: (host). */
MAXE_API maxe_status maxe_handle_tuning(const maxe_handle* h, int32_t* items);

/* a4.  Entropy of the nonzero distribution (Section 4, entropy equation;
 * hierarchical grids of Section 5).  counts[br*gc + bc] is the number of
 * stored entries (i, j) of the handle's matrix with floor(i*gr/rows) = br and
 * floor(j*gc/cols) = bc; H = -sum_{c>0} p log_base p with p = c / nnz
 * (H = 0 when nnz = 0).  1 <= gr <= rows, 1 <= gc <= cols, base > 1.
 * H_host: (host) receives H.  counts_dev: (device) int64[gr*gc] or NULL.
 * alloc: scratch allocator (nullable).  Synchronises `stream`. */
MAXE_API maxe_status maxe_nnz_entropy(const maxe_handle* h, int32_t gr, int32_t gc, double base, double* H_host,
                             int64_t* counts_dev, const maxe_allocator* alloc, void* stream);

/* Hierarchical 2-D entropy map (Section 5: the entropy split into 2x2, 4x4
 * and 8x8 blocks).  The gr x gc count grid (from maxe_nnz_entropy) is cut into
 * L x L blocks, block (a, b) holding grid rows [ceil(a*gr/L), ceil((a+1)*gr/L))
 * and grid columns likewise; H_dev[a*L + b] is the entropy (in `base`) of the
 * counts inside the block, 0 for an empty block.  counts_dev: (device) int64
 * [gr*gc]; H_dev: (device) double [L*L].  1 <= L <= min(gr, gc, 4096).
 * Stream-ordered, no synchronisation; deterministic. */
MAXE_API maxe_status maxe_entropy_levels(const int64_t* counts_dev, int32_t gr, int32_t gc, int32_t L, double base,
                                         double* H_dev, void* stream);

/* Allocation-free form of maxe_nnz_entropy (the paper has no counterpart).
 * Some callers cannot call cudaMalloc: for example a host framework that has
 * reserved all device memory for its own pool and hands a plugin only its
 * input and output buffers, or code on a path where cudaMalloc's implicit
 * device-wide synchronisation is not allowed.  This entry point computes the
 * same counts and H as maxe_nnz_entropy, and allocates nothing: its scratch is
 * a static device array of 65536 32-bit counts plus one double (256 KiB),
 * which every GPU that loads the library holds until the process exits.
 * Arguments as for maxe_nnz_entropy (there is no allocator argument).
 * Limits and behaviour:
 *   - gr * gc must be <= 65536; larger grids return MAXE_ERR_INVALID.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.  The address belongs to the device's context: a call
 *     after the context was destroyed and made anew (cudaDeviceReset) looks
 *     it up again.
 *   - Every call on a device shares the one array and leaves its counts in
 *     it; each call clears the cells it uses before counting.  Calls that
 *     overlap on the GPU (other streams, other host threads) race on the array
 *     and give wrong results: serialise them.
 *   - Synchronises `stream` (H is returned on the host). */
MAXE_API maxe_status maxe_nnz_entropy_noalloc(const maxe_handle* h, int32_t gr, int32_t gc, double base,
                                              double* H_host, int64_t* counts_dev, void* stream);

/* a6 + a5.  y = A x (Section 2, CSR product) through the permuted matrix:
 * without MAXE_VEC_PERMUTED, x is gathered to x' = P_c^{-1} x in handle-owned
 * scratch, y' = A' x' is computed, and y[rperm[i']] = y'[i'] is written in the
 * product's epilogue, so y = A x.  With MAXE_VEC_PERMUTED, y = A' x directly.
 * x: (device) cols elements, y: (device) rows elements; FP64 for MAXE_F64
 * handles, FP32 otherwise.  x and y must not overlap.  Calls on one handle
 * without MAXE_VEC_PERMUTED share its x' scratch: do not overlap them in time. */
MAXE_API maxe_status maxe_spmv(const maxe_handle* h, const void* x, void* y, uint32_t flags, void* stream);

/* a6 + a5 from host memory (Section 2, CSR product): enqueues on `stream`, in
 * this order, the copy of x_host into x_dev, maxe_spmv(h, x_dev, y_dev, flags,
 * stream) and the copy of y_dev into y_host, and returns without waiting:
 * y_host holds y once `stream` has passed the call (synchronise the stream or
 * wait on an event recorded after it).  x_host: (host) cols elements, y_host:
 * (host) rows elements, element type as for maxe_spmv; page-locked host memory
 * lets the copies run asynchronously, while from pageable memory the CUDA
 * driver stages them and the call may block.  x_dev, y_dev: (device) scratch
 * of cols / rows elements owned by the caller, not overlapping each other;
 * x_dev is overwritten.  Flags and the x' scratch as for maxe_spmv.  Errors: INVALID on NULL pointers or unknown flags
 * (nothing enqueued); CUDA when a copy cannot be enqueued. */
MAXE_API maxe_status maxe_spmv_host(const maxe_handle* h, const void* x_host, void* y_host, void* x_dev, void* y_dev,
                                    uint32_t flags, void* stream);

/* f3.  y = A x over the COO form of the handle (Section 2, COO product): the
 * row-sorted triplets of A' in chunks of 256 entries, one warp per chunk,
 * rows that cross chunk edges finished by a second kernel from per-chunk
 * partial sums in chunk order (deterministic).  Vectors, flags and the x'
 * scratch as for maxe_spmv.  Errors: UNSUPPORTED if the handle was created
 * without MAXE_COO; INVALID on NULL pointers or unknown flags. */
MAXE_API maxe_status maxe_coo_spmv(const maxe_handle* h, const void* x, void* y, uint32_t flags, void* stream);

/* The handle's COO row indices: *row = (device) int32[nnz], row[t] = i for the
 * entries t of row i of A' (library-owned, valid until the handle is destroyed).
 * Errors: UNSUPPORTED without MAXE_COO. */
MAXE_API maxe_status maxe_handle_coo(const maxe_handle* h, const int32_t** row);

/* a7.  Y = A X for k right-hand sides (1 <= k <= 64).  X: (device) row-major
 * cols x k with leading dimension ldx >= k; Y: (device) row-major rows x k,
 * ldy >= k.  Element type and flags as for maxe_spmv.  Without
 * MAXE_VEC_PERMUTED, rows of X are gathered into handle-owned scratch.
 * Speed: with 16-byte aligned X and Y and ldx, ldy multiples of 4 (FP32) or 2
 * (FP64), rows are gathered 4 (2) columns per load, also when k is not a
 * multiple (the padding columns of X are read and ignored; Y's are untouched).
 * A handle without nonzeros writes Y = 0 without reading X, which may then be
 * NULL when cols == 0 (the same holds for maxe_spmv's x and y). */
MAXE_API maxe_status maxe_spmm(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y,
                      int64_t ldy, uint32_t flags, void* stream);

/* a9.  Batched persistent SpMV/SpMM (many uneven matrices, each with its own
 * k right-hand sides, in one persistent launch per value type and kernel
 * class present: unit-stride SpMV with 8 or with 16 entries per lane, SpMM by
 * column passes or columns across lanes, or SpMM with one row per lane group
 * for items whose X and Y rows are 16-byte aligned (ldx and ldy multiples of
 * 16 bytes / element size) -- the class maxe_spmm's MAXE_SPMM_ROWS path runs).
 *
 * An item asks for Y = A' X on a handle: X (device) is in the permuted space
 * (x' = x[cperm], rows of X gathered), row-major cols x k with leading
 * dimension ldx >= k; Y (device) rows x k, ldy >= k, written in the permuted
 * space, or through rperm into the original space with MAXE_BATCH_SCATTER_Y.
 * 1 <= k <= 64.  Each handle carries a batch plan (entries per warp task,
 * entries per lane and the SpMM kernel: the handle's own SpMM path when it was
 * autotuned or set by a flag, else one row per lane group), made at creation
 * and retuned by maxe_batch_tune; it does
 * not depend on the other items, so an item's result is bit-identical alone
 * and in any mix.
 *
 * A batch object keeps the descriptor table in pinned host memory and uploads
 * it on the stream right before the launch, so maxe_batch_run can be captured
 * in a CUDA graph (capture after maxe_batch_set; replays use the table as set).
 * A batch object serves one stream at a time; maxe_batch_run waits (on the
 * host) until the previous run's table upload has executed before rewriting
 * the staging. */
#define MAXE_BATCH_SCATTER_Y 0x1u
typedef struct maxe_batch maxe_batch;
typedef struct {
  const maxe_handle* h;
  int32_t k;
  const void* X;
  int64_t ldx;
  void* Y;
  int64_t ldy;
  uint32_t flags; /* 0 or MAXE_BATCH_SCATTER_Y */
} maxe_batch_item;

/* New batch object for up to `capacity` items (1 <= capacity <= 2^20).
 * Device tables come from `alloc` (nullable); the host staging is pinned. */
MAXE_API maxe_status maxe_batch_create(int32_t capacity, const maxe_allocator* alloc, void* stream, maxe_batch** out);
/* Replace the item list (host array of n items, copied).  INVALID on bad items. */
MAXE_API maxe_status maxe_batch_set(maxe_batch* b, const maxe_batch_item* items, int32_t n);
/* Upload the table and launch the persistent kernel(s) on `stream`; the Y of
 * items whose handle has no nonzeros is zeroed by a memset instead (their X is
 * not read). */
MAXE_API maxe_status maxe_batch_run(maxe_batch* b, void* stream);
MAXE_API maxe_status maxe_batch_destroy(maxe_batch* b);
/* Autotune the handle's batch plan for k right-hand sides.  Two batches of
 * copies of the item, whose tasks under the current plan fill the resident
 * warps once and four times over, are timed (the best of three timings each;
 * every plan on the same copies) for: the handle's current plan; entries per task
 * (rows per warp task) in {512, 2048, 8192, 32768} (at least nnz / resident
 * warps) x the kernel variant (8 or 16 entries per lane for k = 1; column
 * passes, columns across lanes or one row per lane group for k > 1); then, for
 * the best of those, the
 * CTA shape of the launch (fewer CTAs per SM than fit).  The current plan is
 * replaced only by one at least 3% faster at both fills, so tuning never keeps
 * a slower plan.  In a batch, a launch uses the largest CTA count per SM its items'
 * plans ask for (all that fit if any item has the default).  Results do not
 * depend on the plan's CTA shape.  Synchronises `stream`. */
MAXE_API maxe_status maxe_batch_tune(maxe_handle* h, int32_t k, void* stream);
/* The handle's batch plan (any output may be NULL). */
MAXE_API maxe_status maxe_batch_plan_info(const maxe_handle* h, int64_t* entries_per_task, int32_t* tasks,
                                          int32_t* items_per_lane);
/* CTAs per SM the handle's batch plan asks of a launch (0: as many as fit). */
MAXE_API maxe_status maxe_batch_plan_shape(const maxe_handle* h, int32_t* blocks_per_sm);

/* Power iteration on a square handle, in the original space (v <- A v / ||A v||_2,
 * `steps` times from v0, then lambda = v^T A v).  Not in the paper: it is the
 * iterative reuse of the matrix that the paper's preconditioning analogy
 * assumes (Section 1).  v0, v_out: (device) rows elements of the handle's
 * vector type; lambda_host: (host).  Synchronises `stream`. */
MAXE_API maxe_status maxe_power_iteration(const maxe_handle* h, const void* v0, int32_t steps, void* v_out,
                                 double* lambda_host, void* stream);

/* maxe_power_iteration that also returns, in lambda_hist_host[s] (host,
 * `steps` doubles), the Rayleigh quotient v_s^T A v_s of the iterate after
 * step s + 1 (the last one equals lambda), taken from the product that starts
 * the next step: no extra products.  Same arguments and errors otherwise
 * (INVALID when lambda_hist_host is NULL). */
MAXE_API maxe_status maxe_power_iteration_history(const maxe_handle* h, const void* v0, int32_t steps,
                                                  void* v_out, double* lambda_host, double* lambda_hist_host,
                                                  void* stream);

/* Vector steps of a batched power iteration kept in the permuted space (used
 * by the serving loop; not in the paper).  With Q = rinv[cperm] (so that
 * u_next = P_c^{-1} P_r^{-1} w for w = A' u), square matrices only:
 *   maxe_vec_norm_gather: nrm2 = sum w[i]^2 (FP64), u[j] = w[Q[j]] / sqrt(nrm2);
 *   maxe_vec_dot_gather:  *out = sum_j u[j] * w[Q[j]] (FP64; the Rayleigh
 *                         quotient v^T A v of the original-space iterate).
 * Q: (device) int32[n] or NULL for the identity; w, u: (device) n elements of
 * elem_bytes (4 = FP32, 8 = FP64); scratch: (device) >= 514 doubles, caller
 * owned; out: (device) one double.  The reductions use a fixed split of the
 * vector, so results are deterministic.  u and w must not overlap. */
MAXE_API maxe_status maxe_vec_norm_gather(const int32_t* Q, int32_t n, int32_t elem_bytes, const void* w, void* u,
                                          double* scratch, void* stream);
MAXE_API maxe_status maxe_vec_dot_gather(const int32_t* Q, int32_t n, int32_t elem_bytes, const void* u,
                                         const void* w, double* scratch, double* out, void* stream);

/* Release a handle and everything it owns (through its allocator, on the
 * stream given at creation).  NULL is accepted. */
MAXE_API maxe_status maxe_handle_destroy(maxe_handle* h);

/* Synchronise `stream`, then return and clear the device-side status:
 * MAXE_ERR_TIMEOUT if a bounded wait ran out since the last call, else MAXE_OK
 * (or MAXE_ERR_CUDA if the stream reported an error). */
MAXE_API maxe_status maxe_device_status(void* stream);

/* Time after which every bounded device-side wait of the library's kernels on
 * the current device gives up (the kernel then records MAXE_ERR_TIMEOUT, stops
 * its work and returns, leaving the context usable).  ns = 0 restores the
 * default of 2 s; at most 60 s (MAXE_ERR_INVALID above).  The limit is a
 * parameter of each launch: it affects kernels launched after the call, and a
 * CUDA graph keeps the limit its kernels were captured with. */
MAXE_API maxe_status maxe_set_wait_limit_ns(uint64_t ns);

/* Self-test of the timeout path: launches on `stream` one small kernel that
 * waits on an mbarrier nothing completes.  Its bounded wait runs out after the
 * wait limit, records the timeout and the kernel returns; the next
 * maxe_device_status(stream) reports MAXE_ERR_TIMEOUT.  Occupies one SM for
 * the wait limit: lower the limit first (maxe_set_wait_limit_ns). */
MAXE_API maxe_status maxe_selftest_wait(void* stream);

/* Human-readable name of a status code. */
MAXE_API const char* maxe_status_str(maxe_status s);

/* Library version as "major.minor.patch". */
MAXE_API const char* maxe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MAXE_H */
