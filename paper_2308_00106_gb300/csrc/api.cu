// api.cu -- the extern "C" entry points of libmaxe.so (declared in include/maxe.h).
// Host-side argument checks, handle lifetime, and dispatch to the kernel
// families; no arithmetic of the method runs here.
#include <atomic>
#include <mutex>
#include <new>

#include "handle.cuh"

namespace maxe {

namespace {
std::atomic<uint64_t> g_wait_ns[64];  // 0: kWaitNs
}  // namespace

uint64_t wait_limit_ns(int device) {
  if (device < 0 || device >= 64) return kWaitNs;
  const uint64_t v = g_wait_ns[device].load(std::memory_order_relaxed);
  return v ? v : kWaitNs;
}

uint64_t wait_limit_ns() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return kWaitNs;
  }
  return wait_limit_ns(dev);
}

maxe_status device_info(DeviceInfo* out) {
  static std::mutex mu;
  static DeviceInfo infos[64];
  static bool ready[64] = {};
  int dev = 0;
  MAXE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MAXE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[dev]) {
    DeviceInfo d{};
    d.device = dev;
    MAXE_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    MAXE_CUDA_TRY(cudaMalloc(&d.status, kDevWordBytes));
    MAXE_CUDA_TRY(cudaMemset(d.status, 0, kDevWordBytes));
    infos[dev] = d;
    ready[dev] = true;
  }
  *out = infos[dev];
  return MAXE_OK;
}

namespace {

// A wait on an mbarrier that nothing completes: it runs out after the wait
// limit, records the timeout and returns (the test of the failure path).
__global__ void selftest_wait_kernel(unsigned* status, uint64_t lim) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, status, lim);
}

}  // namespace

}  // namespace maxe

using namespace maxe;

namespace {

bool bad_size(int64_t n) { return n < 0 || n > kMaxIndex; }
bool bad_dtype(maxe_dtype d) { return d != MAXE_F64 && d != MAXE_F32 && d != MAXE_BF16; }

void release(maxe_handle* h) {
  if (!h) return;
  const Allocator& al = h->al;
  al.put(h->xbuf);
  xslice_release(h);
  al.put(h->coo_carry);
  al.put(h->coo_row);
  al.put(h->bwrow);
  al.put(h->wrow[1]);
  al.put(h->wrow[0]);
  al.put(h->cperm);
  al.put(h->rperm);
  al.put(h->val);
  al.put(h->col);
  al.put(h->rowptr);
  delete h;
}

// x' scratch for k right-hand sides (ld = round_up(k, 4)); grows on demand.
maxe_status ensure_xbuf(maxe_handle* h, int32_t k, cudaStream_t st) {
  if (h->xbuf && h->xbuf_k >= k) return MAXE_OK;
  const int32_t kk = static_cast<int32_t>(round_up(k, 4));
  Allocator al = h->al;
  al.stream = st;
  void* p = al.get(static_cast<size_t>(std::max(h->cols, 1)) * kk * vector_bytes(h->dtype));
  if (!p) return MAXE_ERR_OOM;
  al.put(h->xbuf);
  h->xbuf = p;
  h->xbuf_k = kk;
  return MAXE_OK;
}

}  // namespace

extern "C" {

const char* maxe_status_str(maxe_status s) {
  switch (s) {
    case MAXE_OK: return "MAXE_OK";
    case MAXE_ERR_INVALID: return "MAXE_ERR_INVALID";
    case MAXE_ERR_OOM: return "MAXE_ERR_OOM";
    case MAXE_ERR_CUDA: return "MAXE_ERR_CUDA";
    case MAXE_ERR_TIMEOUT: return "MAXE_ERR_TIMEOUT";
    case MAXE_ERR_UNSUPPORTED: return "MAXE_ERR_UNSUPPORTED";
  }
  return "MAXE_ERR_UNKNOWN";
}

const char* maxe_version(void) { return "0.1.0"; }

maxe_status maxe_build_permutation(uint64_t seed, int32_t n, int32_t tag, int32_t* perm, const maxe_allocator* alloc,
                                   void* stream) {
  if (n < 0 || (tag != 0 && tag != 1) || (n > 0 && !perm)) return MAXE_ERR_INVALID;
  if (n == 0) return MAXE_OK;
  cudaStream_t st = as_stream(stream);
  Allocator al(alloc, st);
  ScratchSet scratch(al);
  uint64_t* keys = scratch.get<uint64_t>(n);
  uint64_t* keys_alt = scratch.get<uint64_t>(n);
  int32_t* vals_alt = scratch.get<int32_t>(n);
  void* rs = scratch.get<unsigned char>(radix_scratch_bytes(n));
  if (!keys || !keys_alt || !vals_alt || !rs) return MAXE_ERR_OOM;
  MAXE_TRY(launch_keys(seed, n, tag, keys, perm, st));
  return radix_sort_pairs(keys, perm, keys_alt, vals_alt, n, 64, rs, st);
}

maxe_status maxe_nnz_histogram(const maxe_csr* A, int32_t axis, int32_t* hist, void* stream) {
  if (!A || (axis != 0 && axis != 1)) return MAXE_ERR_INVALID;
  if (bad_size(A->rows) || bad_size(A->cols) || bad_size(A->nnz) || !A->rowptr) return MAXE_ERR_INVALID;
  if ((axis == 0 ? A->rows : A->cols) > 0 && !hist) return MAXE_ERR_INVALID;
  if (axis == 1 && A->nnz > 0 && !A->col) return MAXE_ERR_INVALID;
  return nnz_histogram_run(A->rowptr, A->col, A->rows, A->cols, A->nnz, axis, hist, as_stream(stream));
}

maxe_status maxe_gradient_permutation(const int32_t* hist, int32_t n, uint64_t seed, int32_t tag, int32_t* perm,
                                      int32_t* pivot, const maxe_allocator* alloc, void* stream) {
  if (n < 0 || (tag != 0 && tag != 1) || (n > 0 && (!hist || !perm))) return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  Allocator al(alloc, st);
  return gradient_permutation_run(hist, n, seed, tag, perm, pivot, al, st);
}

maxe_status maxe_invert_permutation(const int32_t* perm, int32_t n, int32_t* inv, void* stream) {
  if (n < 0 || (n > 0 && (!perm || !inv))) return MAXE_ERR_INVALID;
  return launch_invert(perm, n, inv, as_stream(stream));
}

maxe_status maxe_permute_gather(const int32_t* perm, int32_t n, int32_t elem_bytes, const void* in, void* out,
                                void* stream) {
  if (n < 0 || (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8)) return MAXE_ERR_INVALID;
  if (n > 0 && (!perm || !in || !out)) return MAXE_ERR_INVALID;
  return launch_gather(perm, n, elem_bytes, 1, in, 1, out, 1, as_stream(stream));
}

maxe_status maxe_permute_scatter(const int32_t* perm, int32_t n, int32_t elem_bytes, const void* in, void* out,
                                 void* stream) {
  if (n < 0 || (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8)) return MAXE_ERR_INVALID;
  if (n > 0 && (!perm || !in || !out)) return MAXE_ERR_INVALID;
  return launch_scatter(perm, n, elem_bytes, in, out, as_stream(stream));
}

maxe_status maxe_permute_csr(const maxe_csr* A, const int32_t* rperm, const int32_t* cperm, uint32_t flags,
                             const maxe_allocator* alloc, void* stream, maxe_handle** out) {
  if (!A || !out) return MAXE_ERR_INVALID;
  *out = nullptr;
  if (bad_size(A->rows) || bad_size(A->cols) || bad_size(A->nnz) || bad_dtype(A->dtype)) return MAXE_ERR_INVALID;
  if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return MAXE_ERR_INVALID;
  if (A->nnz > 0 && (A->rows == 0 || A->cols == 0)) return MAXE_ERR_INVALID;
  if (flags & ~static_cast<uint32_t>(MAXE_VALIDATE | MAXE_AUTOTUNE | MAXE_ITEMS16 | MAXE_SPMM_LANES |
                                     MAXE_EQUAL_ROWS | MAXE_COO | MAXE_XSLICE | MAXE_XS_PAIRS | MAXE_XS_SINGLE |
                                     MAXE_SPMM_ROWS | MAXE_SPMM_ROWS_PF))
    return MAXE_ERR_INVALID;
  if ((flags & MAXE_XS_PAIRS) && (flags & MAXE_XS_SINGLE)) return MAXE_ERR_INVALID;
  DeviceInfo di{};
  MAXE_TRY(device_info(&di));
  cudaStream_t st = as_stream(stream);
  maxe_handle* h = new (std::nothrow) maxe_handle();
  if (!h) return MAXE_ERR_OOM;
  h->rows = A->rows;
  h->cols = A->cols;
  h->nnz = A->nnz;
  h->dtype = A->dtype;
  h->al = Allocator(alloc, st);
  h->device = di.device;
  h->sms = di.sms;
  h->status = di.status;
  h->equal_rows = (flags & MAXE_EQUAL_ROWS) ? 1 : 0;
  maxe_status s = permute_csr_run(A, rperm, cperm, flags, h, st);
  if (s == MAXE_OK) s = ensure_xbuf(h, 1, st);
  if (s == MAXE_OK && (flags & MAXE_COO)) s = coo_build(h, st);
  if (s == MAXE_OK && (flags & (MAXE_XSLICE | MAXE_AUTOTUNE)) && !h->equal_rows) {
    const int pairs = (flags & MAXE_XS_PAIRS) ? 1 : ((flags & MAXE_XS_SINGLE) ? -1 : 0);
    s = xslice_build(h, st, (flags & MAXE_XSLICE) != 0, pairs);
    // only the autotuner asked for it: without the memory, the handle goes without it
    if (s == MAXE_ERR_OOM && !(flags & MAXE_XSLICE)) {
      xslice_release(h);
      s = MAXE_OK;
    }
  }
  if (s == MAXE_OK) s = batch_plan_default(h, st);
  if (s == MAXE_OK && (flags & MAXE_ITEMS16)) h->spmv_items16 = 1;
  if (s == MAXE_OK && (flags & MAXE_SPMM_LANES)) h->spmm_lc = 1;
  if (s == MAXE_OK && (flags & MAXE_SPMM_ROWS)) h->spmm_rows = 1;
  if (s == MAXE_OK && (flags & MAXE_SPMM_ROWS_PF)) h->spmm_rows_pf = 1;
  if (s == MAXE_OK && (flags & MAXE_AUTOTUNE)) s = spmv_autotune(h, st);
  // the default batch plan follows the handle's SpMM path where it was tuned
  // or asked for, else takes the rows kernel
  if (s == MAXE_OK) h->blc = h->spmm_rows ? 2 : (h->spmm_lc ? 1 : ((flags & MAXE_AUTOTUNE) ? 0 : 2));
  if (s != MAXE_OK) {
    release(h);
    return s;
  }
  *out = h;
  return MAXE_OK;
}

maxe_status maxe_handle_csr(const maxe_handle* h, maxe_csr* view, const int32_t** rperm, const int32_t** cperm) {
  if (!h || !view) return MAXE_ERR_INVALID;
  view->rows = h->rows;
  view->cols = h->cols;
  view->nnz = h->nnz;
  view->rowptr = h->rowptr;
  view->col = h->col;
  view->val = h->val;
  view->dtype = h->dtype;
  if (rperm) *rperm = h->rperm;
  if (cperm) *cperm = h->cperm;
  return MAXE_OK;
}

maxe_status maxe_handle_tuning(const maxe_handle* h, int32_t* items) {
  if (!h || !items) return MAXE_ERR_INVALID;
  *items = (h->spmv_items16 ? 16 : 8) | (h->spmm_lc ? 0x100 : 0) | (h->xs_use ? 0x200 : 0) |
           (h->xs_use && h->xs_prefetch ? 0x400 : 0) | (h->xs_use && h->xs_pair == 2 ? 0x800 : 0) |
           (h->spmm_rows ? 0x1000 : 0) | ((h->blc & 3) << 13) | (((h->xs_ahead / 512) & 7) << 15) |
           (h->spmm_rows_pf ? 0x40000 : 0);
  return MAXE_OK;
}

maxe_status maxe_nnz_entropy(const maxe_handle* h, int32_t gr, int32_t gc, double base, double* H_host,
                             int64_t* counts_dev, const maxe_allocator* alloc, void* stream) {
  if (!h || !H_host) return MAXE_ERR_INVALID;
  if (gr < 1 || gc < 1 || gr > h->rows || gc > h->cols || !(base > 1.0)) return MAXE_ERR_INVALID;
  if (static_cast<int64_t>(gr) * gc > (int64_t(1) << 31)) return MAXE_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  return entropy_run(h, gr, gc, base, H_host, counts_dev, Allocator(alloc, st), st);
}

maxe_status maxe_spmv(const maxe_handle* h, const void* x, void* y, uint32_t flags, void* stream) {
  if (!h || flags & ~static_cast<uint32_t>(MAXE_VEC_PERMUTED)) return MAXE_ERR_INVALID;
  if ((h->cols > 0 && !x) || (h->rows > 0 && !y)) return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  if (flags & MAXE_VEC_PERMUTED) return spmm_launch(h, 1, x, 1, y, 1, nullptr, st);
  const void* xs = x;
  if (h->cperm) {
    MAXE_TRY(launch_gather(h->cperm, h->cols, vector_bytes(h->dtype), 1, x, 1, h->xbuf, 1, st));
    xs = h->xbuf;
  }
  return spmm_launch(h, 1, xs, 1, y, 1, h->rperm, st);
}

maxe_status maxe_spmv_host(const maxe_handle* h, const void* x_host, void* y_host, void* x_dev, void* y_dev,
                           uint32_t flags, void* stream) {
  if (!h || flags & ~static_cast<uint32_t>(MAXE_VEC_PERMUTED)) return MAXE_ERR_INVALID;
  if ((h->cols > 0 && (!x_host || !x_dev)) || (h->rows > 0 && (!y_host || !y_dev))) return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  const size_t eb = vector_bytes(h->dtype);
  if (h->cols > 0)
    MAXE_CUDA_TRY(cudaMemcpyAsync(x_dev, x_host, eb * static_cast<size_t>(h->cols), cudaMemcpyHostToDevice, st));
  MAXE_TRY(maxe_spmv(h, x_dev, y_dev, flags, stream));
  if (h->rows > 0)
    MAXE_CUDA_TRY(cudaMemcpyAsync(y_host, y_dev, eb * static_cast<size_t>(h->rows), cudaMemcpyDeviceToHost, st));
  return MAXE_OK;
}

maxe_status maxe_coo_spmv(const maxe_handle* h, const void* x, void* y, uint32_t flags, void* stream) {
  if (!h || flags & ~static_cast<uint32_t>(MAXE_VEC_PERMUTED)) return MAXE_ERR_INVALID;
  if ((h->cols > 0 && !x) || (h->rows > 0 && !y)) return MAXE_ERR_INVALID;
  if (!h->coo_row) return MAXE_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  if (flags & MAXE_VEC_PERMUTED) return coo_spmv_launch(h, x, y, nullptr, st);
  const void* xs = x;
  if (h->cperm) {
    MAXE_TRY(launch_gather(h->cperm, h->cols, vector_bytes(h->dtype), 1, x, 1, h->xbuf, 1, st));
    xs = h->xbuf;
  }
  return coo_spmv_launch(h, xs, y, h->rperm, st);
}

maxe_status maxe_handle_coo(const maxe_handle* h, const int32_t** row) {
  if (!h || !row) return MAXE_ERR_INVALID;
  *row = h->coo_row;
  return h->coo_row ? MAXE_OK : MAXE_ERR_UNSUPPORTED;
}

maxe_status maxe_spmm(const maxe_handle* h, int32_t k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                      uint32_t flags, void* stream) {
  if (!h || k < 1 || k > 64 || ldx < k || ldy < k) return MAXE_ERR_INVALID;
  if (flags & ~static_cast<uint32_t>(MAXE_VEC_PERMUTED)) return MAXE_ERR_INVALID;
  if ((h->cols > 0 && !X) || (h->rows > 0 && !Y)) return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  if (flags & MAXE_VEC_PERMUTED) return spmm_launch(h, k, X, ldx, Y, ldy, nullptr, st);
  const void* xs = X;
  int64_t lds = ldx;
  if (h->cperm) {
    maxe_handle* hm = const_cast<maxe_handle*>(h);
    MAXE_TRY(ensure_xbuf(hm, k, st));
    lds = hm->xbuf_k;
    MAXE_TRY(launch_gather(h->cperm, h->cols, vector_bytes(h->dtype), k, X, ldx, hm->xbuf, lds, st));
    xs = hm->xbuf;
  }
  return spmm_launch(h, k, xs, lds, Y, ldy, h->rperm, st);
}

maxe_status maxe_power_iteration(const maxe_handle* h, const void* v0, int32_t steps, void* v_out,
                                 double* lambda_host, void* stream) {
  if (!h || !lambda_host || steps < 0 || h->rows != h->cols) return MAXE_ERR_INVALID;
  if (h->rows > 0 && (!v0 || !v_out)) return MAXE_ERR_INVALID;
  return power_iteration_run(h, v0, steps, v_out, lambda_host, nullptr, as_stream(stream));
}

maxe_status maxe_power_iteration_history(const maxe_handle* h, const void* v0, int32_t steps, void* v_out,
                                         double* lambda_host, double* lambda_hist_host, void* stream) {
  if (!h || !lambda_host || !lambda_hist_host || steps < 0 || h->rows != h->cols) return MAXE_ERR_INVALID;
  if (h->rows > 0 && (!v0 || !v_out)) return MAXE_ERR_INVALID;
  return power_iteration_run(h, v0, steps, v_out, lambda_host, lambda_hist_host, as_stream(stream));
}

maxe_status maxe_handle_destroy(maxe_handle* h) {
  release(h);
  return MAXE_OK;
}

maxe_status maxe_set_wait_limit_ns(uint64_t ns) {
  if (ns > 60000000000ull) return MAXE_ERR_INVALID;
  DeviceInfo di{};
  MAXE_TRY(device_info(&di));
  g_wait_ns[di.device].store(ns, std::memory_order_relaxed);
  return MAXE_OK;
}

maxe_status maxe_selftest_wait(void* stream) {
  DeviceInfo di{};
  MAXE_TRY(device_info(&di));
  selftest_wait_kernel<<<1, 32, 0, as_stream(stream)>>>(di.status, wait_limit_ns(di.device));
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

maxe_status maxe_device_status(void* stream) {
  DeviceInfo di{};
  MAXE_TRY(device_info(&di));
  cudaStream_t st = as_stream(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return MAXE_ERR_CUDA;
  unsigned v = 0;
  MAXE_CUDA_TRY(cudaMemcpy(&v, di.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (v) MAXE_CUDA_TRY(cudaMemset(di.status, 0, sizeof(unsigned)));
  return (v & kDevTimeout) ? MAXE_ERR_TIMEOUT : MAXE_OK;
}

}  // extern "C"
