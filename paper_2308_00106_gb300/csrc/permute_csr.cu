// permute_csr.cu -- build A' = P_r A P_c (Eq. 1) in CSR with ascending columns
// (Section 2), values copied bit for bit.
//
//   1. len'[i'] = len(rperm[i'])                      (gather of row lengths)
//   2. rowptr' = exclusive scan of len'               (scan.cu)
//   3. bucket the new rows by where they start (buckets of kBucket = 2048
//      entries).  One CTA per bucket gathers the entries of its rows from the
//      old matrix, relabels each column c -> cinv[c], and sorts the bucket in
//      shared memory by the 55-bit key (row start | new column | position),
//      which sorts each row by new column and keeps equal columns in their old
//      order.  A bucket holds < 4096 entries as long as no row in it is longer
//      than kLong = 2048.
//   4. rows longer than kLong (the paper's dense-row case, Section 1) are
//      gathered into one list keyed by (long-row id, new column) and sorted
//      with the radix sort of perm.cu, then written to their rows.
#include <algorithm>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kBucket = 2048;
constexpr int kLong = 2048;
constexpr int kSortCap = 4096;  // entries per bucket tile
constexpr int kRowsCap = 4096;  // rows of a bucket held in shared memory
constexpr int kSortThreads = 512;

__global__ void row_lengths_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ rperm, int32_t M,
                                   int32_t* __restrict__ len) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int32_t r = rperm ? rperm[i] : static_cast<int32_t>(i);
  len[i] = rowptr[r + 1] - rowptr[r];
}

template <typename VT>
struct SortSmem {
  uint64_t keys[kSortCap];
  VT vals[kSortCap];
  int32_t rstart[kRowsCap + 1];  // new row starts, local to the bucket
  int32_t ostart[kRowsCap];      // old row starts
};

// One CTA per bucket g: rows [first[g], first[g+1]) minus a trailing long row.
template <typename VT>
__global__ void __launch_bounds__(kSortThreads) bucket_sort_kernel(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const int32_t* __restrict__ rperm, const int32_t* __restrict__ cinv, const int32_t* __restrict__ nrowptr,
    const int32_t* __restrict__ first, int32_t M, int64_t Z, int32_t* __restrict__ ncol, VT* __restrict__ nval) {
  extern __shared__ __align__(16) unsigned char raw[];
  SortSmem<VT>& sm = *reinterpret_cast<SortSmem<VT>*>(raw);
  const int g = blockIdx.x;
  const int32_t r0 = first[g], r1 = first[g + 1];
  if (r0 >= r1) return;
  int32_t rhi = r1;
  const int64_t base = nrowptr[r0];
  int64_t end = (r1 < M) ? static_cast<int64_t>(nrowptr[r1]) : Z;
  if (nrowptr[r1 - 1] + static_cast<int64_t>(kLong) < end) {  // trailing long row: handled elsewhere
    rhi = r1 - 1;
    end = nrowptr[r1 - 1];
  }
  const int count = static_cast<int>(end - base);
  if (count <= 0) return;
  const int nrows = rhi - r0;
  const bool rows_in_smem = nrows <= kRowsCap;
  if (rows_in_smem) {
    for (int t = threadIdx.x; t < nrows; t += kSortThreads) {
      const int32_t r = r0 + t;
      sm.rstart[t] = static_cast<int32_t>(nrowptr[r] - base);
      sm.ostart[t] = rowptr[rperm ? rperm[r] : r];
    }
  }
  __syncthreads();
  int sz = 1;
  while (sz < count) sz <<= 1;
  for (int pos = threadIdx.x; pos < sz; pos += kSortThreads) {
    if (pos >= count) {
      sm.keys[pos] = ~0ull;
      continue;
    }
    // row containing entry pos: last row whose start <= pos
    int lo = 0, hi = nrows - 1;
    int32_t rs, os;
    if (rows_in_smem) {
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sm.rstart[mid] <= pos) lo = mid; else hi = mid - 1;
      }
      rs = sm.rstart[lo];
      os = sm.ostart[lo];
    } else {
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nrowptr[r0 + mid] - base <= pos) lo = mid; else hi = mid - 1;
      }
      const int32_t r = r0 + lo;
      rs = static_cast<int32_t>(nrowptr[r] - base);
      os = rowptr[rperm ? rperm[r] : r];
    }
    const int64_t src = static_cast<int64_t>(os) + (pos - rs);
    const int32_t c = col[src];
    const uint32_t nc = static_cast<uint32_t>(cinv ? cinv[c] : c);
    sm.keys[pos] = (static_cast<uint64_t>(rs) << 43) | (static_cast<uint64_t>(nc) << 12) | static_cast<uint64_t>(pos);
    sm.vals[pos] = val[src];
  }
  __syncthreads();
  // bitonic sort of sz keys
  for (int kk = 2; kk <= sz; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (sz >> 1); t += kSortThreads) {
        const int lo_i = 2 * t - (t & (j - 1));
        const int hi_i = lo_i + j;
        const bool up = (lo_i & kk) == 0;
        const uint64_t a = sm.keys[lo_i], b = sm.keys[hi_i];
        if ((a > b) == up) {
          sm.keys[lo_i] = b;
          sm.keys[hi_i] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int pos = threadIdx.x; pos < count; pos += kSortThreads) {
    const uint64_t key = sm.keys[pos];
    ncol[base + pos] = static_cast<int32_t>((key >> 12) & 0x7FFFFFFFull);
    nval[base + pos] = sm.vals[key & 0xFFFull];
  }
}

__global__ void long_flags_kernel(const int32_t* __restrict__ len, int32_t M, int32_t* __restrict__ flag,
                                  unsigned long long* __restrict__ stats) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int isl = len[i] > kLong;
  flag[i] = isl;
  if (isl) {
    atomicAdd(&stats[0], 1ull);
    atomicAdd(&stats[1], static_cast<unsigned long long>(len[i]));
  }
}

__global__ void long_compact_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ ids, int32_t M,
                                    const int32_t* __restrict__ len, int32_t* __restrict__ rows,
                                    int32_t* __restrict__ lens) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M || !flag[i]) return;
  rows[ids[i]] = static_cast<int32_t>(i);
  lens[ids[i]] = len[i];
}

// One CTA per long row: key = (id << colbits) | new column, value = old entry index.
__global__ void long_fill_kernel(const int32_t* __restrict__ lrows, const int32_t* __restrict__ seg,
                                 const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ rperm, const int32_t* __restrict__ cinv, int colbits,
                                 uint64_t* __restrict__ keys, int32_t* __restrict__ src) {
  const int id = blockIdx.x;
  const int32_t r = lrows[id];
  const int32_t o = rowptr[rperm ? rperm[r] : r];
  const int32_t n = rowptr[(rperm ? rperm[r] : r) + 1] - o;
  const int64_t s0 = seg[id];
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int32_t c = col[o + t];
    const uint64_t nc = static_cast<uint64_t>(cinv ? cinv[c] : c);
    keys[s0 + t] = (static_cast<uint64_t>(id) << colbits) | nc;
    src[s0 + t] = o + t;
  }
}

template <typename VT>
__global__ void long_write_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ src, int64_t n,
                                  int colbits, const int32_t* __restrict__ seg, const int32_t* __restrict__ lrows,
                                  const int32_t* __restrict__ nrowptr, const VT* __restrict__ val,
                                  int32_t* __restrict__ ncol, VT* __restrict__ nval) {
  const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint64_t key = keys[s];
  const int id = static_cast<int>(key >> colbits);
  const int64_t dst = static_cast<int64_t>(nrowptr[lrows[id]]) + (s - seg[id]);
  ncol[dst] = static_cast<int32_t>(key & ((1ull << colbits) - 1));
  nval[dst] = val[src[s]];
}

// Validation (MAXE_VALIDATE): any failure sets *bad.
__global__ void validate_csr_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t M,
                                    int32_t N, int64_t Z, int* __restrict__ bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i == 0 && (rowptr[0] != 0 || rowptr[M] != Z)) atomicOr(bad, 1);
  if (i < M && rowptr[i + 1] < rowptr[i]) atomicOr(bad, 1);
  if (i < Z && (col[i] < 0 || col[i] >= N)) atomicOr(bad, 1);
}

__global__ void count_perm_kernel(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ seen,
                                  int* __restrict__ bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t p = perm[i];
  if (p < 0 || p >= n || atomicAdd(&seen[p], 1) != 0) atomicOr(bad, 1);
}

inline unsigned grid_for(int64_t n, int b = 256) { return static_cast<unsigned>(std::max<int64_t>(1, ceil_div(n, b))); }

template <typename VT>
maxe_status bucket_sort_launch(const maxe_csr* A, const int32_t* rperm, const int32_t* cinv, maxe_handle* h,
                               const int32_t* first, int64_t nb, cudaStream_t st) {
  auto kern = bucket_sort_kernel<VT>;
  const size_t smem = sizeof(SortSmem<VT>);
  MAXE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  kern<<<static_cast<unsigned>(nb), kSortThreads, smem, st>>>(A->rowptr, A->col, static_cast<const VT*>(A->val),
                                                               rperm, cinv, h->rowptr, first, A->rows, A->nnz,
                                                               h->col, static_cast<VT*>(h->val));
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename VT>
maxe_status long_write_launch(const uint64_t* keys, const int32_t* src, int64_t n, int colbits, const int32_t* seg,
                              const int32_t* lrows, maxe_handle* h, const void* val, cudaStream_t st) {
  long_write_kernel<VT><<<grid_for(n), 256, 0, st>>>(keys, src, n, colbits, seg, lrows, h->rowptr,
                                                     static_cast<const VT*>(val), h->col, static_cast<VT*>(h->val));
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

int bits_for(int64_t n) {  // bits to hold values 0..n-1 (at least 1)
  int b = 1;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

}  // namespace

maxe_status permute_csr_run(const maxe_csr* A, const int32_t* rperm, const int32_t* cperm, uint32_t flags,
                            maxe_handle* h, cudaStream_t st) {
  const int32_t M = A->rows, N = A->cols;
  const int64_t Z = A->nnz;
  const Allocator& al = h->al;
  ScratchSet scratch(al);

  if (flags & MAXE_VALIDATE) {
    int* bad = scratch.get<int>(1);
    int32_t* seen = scratch.get<int32_t>(static_cast<size_t>(std::max<int64_t>(std::max(M, N), 1)));
    if (!bad || !seen) return MAXE_ERR_OOM;
    MAXE_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    validate_csr_kernel<<<grid_for(std::max<int64_t>(M + 1, Z)), 256, 0, st>>>(A->rowptr, A->col, M, N, Z, bad);
    if (rperm) {
      MAXE_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(int32_t) * M, st));
      count_perm_kernel<<<grid_for(M), 256, 0, st>>>(rperm, M, seen, bad);
    }
    if (cperm) {
      MAXE_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(int32_t) * N, st));
      count_perm_kernel<<<grid_for(N), 256, 0, st>>>(cperm, N, seen, bad);
    }
    MAXE_CUDA_TRY(cudaGetLastError());
    int hbad = 0;
    MAXE_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    MAXE_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) return MAXE_ERR_INVALID;
  }

  // owned arrays
  const int vb = value_bytes(A->dtype);
  h->nnz_pad = round_up(Z + spmv_pad_elems(), kPadElems);
  h->rowptr = static_cast<int32_t*>(al.get(static_cast<size_t>(M + 1 + kRowptrPad) * sizeof(int32_t)));
  h->col = static_cast<int32_t*>(al.get(static_cast<size_t>(h->nnz_pad) * sizeof(int32_t)));
  h->val = al.get(static_cast<size_t>(h->nnz_pad) * vb);
  if (!h->rowptr || !h->col || !h->val) return MAXE_ERR_OOM;
  MAXE_CUDA_TRY(cudaMemsetAsync(h->rowptr + M, 0, (1 + kRowptrPad) * sizeof(int32_t), st));
  MAXE_CUDA_TRY(cudaMemsetAsync(h->col + Z, 0, (h->nnz_pad - Z) * sizeof(int32_t), st));
  MAXE_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(h->val) + Z * vb, 0, (h->nnz_pad - Z) * vb, st));
  if (rperm) {
    h->rperm = static_cast<int32_t*>(al.get(static_cast<size_t>(std::max(M, 1)) * sizeof(int32_t)));
    if (!h->rperm) return MAXE_ERR_OOM;
    MAXE_CUDA_TRY(cudaMemcpyAsync(h->rperm, rperm, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
  }
  if (cperm) {
    h->cperm = static_cast<int32_t*>(al.get(static_cast<size_t>(std::max(N, 1)) * sizeof(int32_t)));
    if (!h->cperm) return MAXE_ERR_OOM;
    MAXE_CUDA_TRY(cudaMemcpyAsync(h->cperm, cperm, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
  }

  if (M > 0) {
    // 1-2. new row pointers
    int32_t* scan_tmp = scratch.get<int32_t>(scan_scratch_elems(M));
    int32_t* cinv = nullptr;
    if (cperm) {
      cinv = scratch.get<int32_t>(static_cast<size_t>(std::max(N, 1)));
      if (!cinv) return MAXE_ERR_OOM;
      MAXE_TRY(launch_invert(cperm, N, cinv, st));
    }
    if (!scan_tmp) return MAXE_ERR_OOM;
    row_lengths_kernel<<<grid_for(M), 256, 0, st>>>(A->rowptr, rperm, M, h->rowptr);
    MAXE_CUDA_TRY(cudaGetLastError());
    // keep the lengths for the long-row pass before scanning in place
    int32_t* len = scratch.get<int32_t>(static_cast<size_t>(M));
    if (!len) return MAXE_ERR_OOM;
    MAXE_CUDA_TRY(cudaMemcpyAsync(len, h->rowptr, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
    MAXE_TRY(scan_exclusive_i32(h->rowptr, h->rowptr, M, h->rowptr + M, scan_tmp, st));

    if (Z > 0) {
      // 3. buckets of short rows
      const int64_t nb = ceil_div(Z, kBucket);
      int32_t* first = scratch.get<int32_t>(static_cast<size_t>(nb + 1));
      if (!first) return MAXE_ERR_OOM;
      MAXE_TRY(bucket_lower_bounds(h->rowptr, M, kBucket, 0, nb, first, st));
      switch (A->dtype) {
        case MAXE_F64: MAXE_TRY(bucket_sort_launch<uint64_t>(A, rperm, cinv, h, first, nb, st)); break;
        case MAXE_F32: MAXE_TRY(bucket_sort_launch<uint32_t>(A, rperm, cinv, h, first, nb, st)); break;
        case MAXE_BF16: MAXE_TRY(bucket_sort_launch<uint16_t>(A, rperm, cinv, h, first, nb, st)); break;
      }

      // 4. long rows
      int32_t* lflag = scratch.get<int32_t>(static_cast<size_t>(M));
      unsigned long long* stats = scratch.get<unsigned long long>(2);
      if (!lflag || !stats) return MAXE_ERR_OOM;
      MAXE_CUDA_TRY(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st));
      long_flags_kernel<<<grid_for(M), 256, 0, st>>>(len, M, lflag, stats);
      MAXE_CUDA_TRY(cudaGetLastError());
      unsigned long long hs[2] = {0, 0};
      MAXE_CUDA_TRY(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
      MAXE_CUDA_TRY(cudaStreamSynchronize(st));
      const int64_t nlong = static_cast<int64_t>(hs[0]), tlong = static_cast<int64_t>(hs[1]);
      if (nlong > 0) {
        int32_t* ids = scratch.get<int32_t>(static_cast<size_t>(M));
        int32_t* lrows = scratch.get<int32_t>(static_cast<size_t>(nlong));
        int32_t* llen = scratch.get<int32_t>(static_cast<size_t>(nlong + 1));
        int32_t* scan2 = scratch.get<int32_t>(scan_scratch_elems(std::max<int64_t>(M, nlong)));
        if (!ids || !lrows || !llen || !scan2) return MAXE_ERR_OOM;
        MAXE_TRY(scan_exclusive_i32(lflag, ids, M, nullptr, scan2, st));
        long_compact_kernel<<<grid_for(M), 256, 0, st>>>(lflag, ids, M, len, lrows, llen);
        MAXE_CUDA_TRY(cudaGetLastError());
        MAXE_TRY(scan_exclusive_i32(llen, llen, nlong, llen + nlong, scan2, st));  // llen -> segment starts
        const int colbits = bits_for(N);
        const int idbits = bits_for(nlong);
        if (colbits + idbits > 64) return MAXE_ERR_UNSUPPORTED;
        // radix sort buffers (own allocations: the scratch set holds at most 16)
        uint64_t* k0 = static_cast<uint64_t*>(al.get(sizeof(uint64_t) * tlong));
        uint64_t* k1 = static_cast<uint64_t*>(al.get(sizeof(uint64_t) * tlong));
        int32_t* v0 = static_cast<int32_t*>(al.get(sizeof(int32_t) * tlong));
        int32_t* v1 = static_cast<int32_t*>(al.get(sizeof(int32_t) * tlong));
        void* rs = al.get(radix_scratch_bytes(tlong));
        maxe_status stt = (k0 && k1 && v0 && v1 && rs) ? MAXE_OK : MAXE_ERR_OOM;
        if (stt == MAXE_OK) {
          long_fill_kernel<<<static_cast<unsigned>(nlong), 256, 0, st>>>(lrows, llen, A->rowptr, A->col, rperm, cinv,
                                                                         colbits, k0, v0);
          stt = cudaGetLastError() == cudaSuccess ? MAXE_OK : MAXE_ERR_CUDA;
        }
        if (stt == MAXE_OK) stt = radix_sort_pairs(k0, v0, k1, v1, tlong, colbits + idbits, rs, st);
        if (stt == MAXE_OK) {
          switch (A->dtype) {
            case MAXE_F64: stt = long_write_launch<uint64_t>(k0, v0, tlong, colbits, llen, lrows, h, A->val, st); break;
            case MAXE_F32: stt = long_write_launch<uint32_t>(k0, v0, tlong, colbits, llen, lrows, h, A->val, st); break;
            case MAXE_BF16: stt = long_write_launch<uint16_t>(k0, v0, tlong, colbits, llen, lrows, h, A->val, st); break;
          }
        }
        al.put(rs);
        al.put(v1);
        al.put(v0);
        al.put(k1);
        al.put(k0);
        if (stt != MAXE_OK) return stt;
      }
    }
  } else {
    MAXE_CUDA_TRY(cudaMemsetAsync(h->rowptr, 0, sizeof(int32_t), st));
  }
  return spmv_build_partition(h, st);
}

}  // namespace maxe
