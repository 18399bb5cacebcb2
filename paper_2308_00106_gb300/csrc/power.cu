// power.cu -- power iteration v <- A v / ||A v||_2 on a handle, in the original
// space (the permuted product of Eq. 1 with x gathered through cperm and y
// scattered through rperm).  Not in the paper: it is the reuse of one matrix
// across many products that the paper's preconditioning analogy (Section 1)
// assumes, and the serving loop's iterative request type.
//
// Norms and the Rayleigh quotient are FP64 two-stage reductions with a fixed
// block split, so the result is deterministic.  The normalisation reads the
// norm from device memory: no host round trip inside the loop.
#include <algorithm>

#include "handle.cuh"

namespace maxe {
namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 512;

template <typename T>
__global__ void __launch_bounds__(kDotThreads) dot_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                           int64_t n, double* __restrict__ part) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = std::min<int64_t>(n, lo + per);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kDotThreads)
    acc += static_cast<double>(a[i]) * static_cast<double>(b[i]);
  __shared__ double ws[kDotThreads / 32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void dot_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    *out = t;
  }
}

template <typename T>
__global__ void scale_by_inv_norm(const T* __restrict__ w, const double* __restrict__ nrm2, int64_t n,
                                  T* __restrict__ v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double inv = 1.0 / sqrt(*nrm2);
  v[i] = static_cast<T>(static_cast<double>(w[i]) * inv);
}

// out[j] = w[Q[j]] * (1 / sqrt(*nrm2))
template <typename T>
__global__ void gather_scale(const int32_t* __restrict__ Q, const T* __restrict__ w, const double* __restrict__ nrm2,
                             int64_t n, T* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double inv = 1.0 / sqrt(*nrm2);
  const int64_t src = Q ? static_cast<int64_t>(Q[i]) : i;
  out[i] = static_cast<T>(static_cast<double>(w[src]) * inv);
}

// part[b] = sum over block b's slice of u[i] * w[Q[i]]
template <typename T>
__global__ void __launch_bounds__(kDotThreads) dot_gather_partial(const T* __restrict__ u, const T* __restrict__ w,
                                                                  const int32_t* __restrict__ Q, int64_t n,
                                                                  double* __restrict__ part) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = std::min<int64_t>(n, lo + per);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kDotThreads)
    acc += static_cast<double>(u[i]) * static_cast<double>(w[Q ? static_cast<int64_t>(Q[i]) : i]);
  __shared__ double ws[kDotThreads / 32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kDotThreads / 32; ++k) t += ws[k];
    part[blockIdx.x] = t;
  }
}

template <typename T>
maxe_status dot(const T* a, const T* b, int64_t n, double* part, double* out, cudaStream_t st) {
  const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kDotBlocks, ceil_div(n, 4 * kDotThreads))));
  dot_partial<T><<<nb, kDotThreads, 0, st>>>(a, b, n, part);
  dot_final<<<1, 32, 0, st>>>(part, nb, out);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

// hist_host (nullable): the Rayleigh quotient v^T A v of the iterate after
// every step, taken from the product that starts the next step (no extra
// products); the last one is lambda.
template <typename T>
maxe_status run(const maxe_handle* h, const T* v0, int32_t steps, T* v, double* lambda_host, double* hist_host,
                cudaStream_t st) {
  const int64_t n = h->rows;
  ScratchSet scratch(h->al);
  T* w = scratch.get<T>(static_cast<size_t>(n));
  T* xp = scratch.get<T>(static_cast<size_t>(n));
  double* part = scratch.get<double>(kDotBlocks + 2 + (hist_host ? std::max(steps, 1) : 0));
  if (!w || !xp || !part) return MAXE_ERR_OOM;
  double* nrm2 = part + kDotBlocks;
  double* lam = part + kDotBlocks + 1;
  double* hist = hist_host ? part + kDotBlocks + 2 : nullptr;
  MAXE_CUDA_TRY(cudaMemcpyAsync(v, v0, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, ceil_div(n, 256)));
  auto product = [&](const T* x, T* y) -> maxe_status {
    const T* xs = x;
    if (h->cperm) {
      MAXE_TRY(launch_gather(h->cperm, n, sizeof(T), 1, x, 1, xp, 1, st));
      xs = xp;
    }
    return spmm_launch(h, 1, xs, 1, y, 1, h->rperm, st);
  };
  for (int32_t s = 0; s < steps; ++s) {
    MAXE_TRY(product(v, w));
    if (hist && s > 0) MAXE_TRY(dot(v, w, n, part, hist + s - 1, st));  // v = the iterate after step s
    MAXE_TRY(dot(w, w, n, part, nrm2, st));
    scale_by_inv_norm<T><<<grid, 256, 0, st>>>(w, nrm2, n, v);
    MAXE_CUDA_TRY(cudaGetLastError());
  }
  MAXE_TRY(product(v, w));
  MAXE_TRY(dot(v, w, n, part, lam, st));
  MAXE_CUDA_TRY(cudaMemcpyAsync(lambda_host, lam, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (hist && steps > 0) {
    if (steps > 1)
      MAXE_CUDA_TRY(cudaMemcpyAsync(hist_host, hist, sizeof(double) * (steps - 1), cudaMemcpyDeviceToHost, st));
    MAXE_CUDA_TRY(cudaMemcpyAsync(hist_host + steps - 1, lam, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  MAXE_CUDA_TRY(cudaStreamSynchronize(st));
  return MAXE_OK;
}

int dot_blocks(int64_t n) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kDotBlocks, ceil_div(n, 4 * kDotThreads))));
}

template <typename T>
maxe_status norm_gather(const int32_t* Q, int64_t n, const T* w, T* u, double* scratch, cudaStream_t st) {
  const int nb = dot_blocks(n);
  dot_partial<T><<<nb, kDotThreads, 0, st>>>(w, w, n, scratch);
  dot_final<<<1, 32, 0, st>>>(scratch, nb, scratch + kDotBlocks);
  gather_scale<T><<<static_cast<unsigned>(std::max<int64_t>(1, ceil_div(n, 256))), 256, 0, st>>>(
      Q, w, scratch + kDotBlocks, n, u);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

template <typename T>
maxe_status dot_gather(const int32_t* Q, int64_t n, const T* u, const T* w, double* scratch, double* out,
                       cudaStream_t st) {
  const int nb = dot_blocks(n);
  dot_gather_partial<T><<<nb, kDotThreads, 0, st>>>(u, w, Q, n, scratch);
  dot_final<<<1, 32, 0, st>>>(scratch, nb, out);
  MAXE_CUDA_TRY(cudaGetLastError());
  return MAXE_OK;
}

}  // namespace

maxe_status power_iteration_run(const maxe_handle* h, const void* v0, int32_t steps, void* v_out,
                                double* lambda_host, double* hist_host, cudaStream_t st) {
  if (h->dtype == MAXE_F64)
    return run<double>(h, static_cast<const double*>(v0), steps, static_cast<double*>(v_out), lambda_host, hist_host,
                       st);
  return run<float>(h, static_cast<const float*>(v0), steps, static_cast<float*>(v_out), lambda_host, hist_host, st);
}

}  // namespace maxe

extern "C" {

maxe_status maxe_vec_norm_gather(const int32_t* Q, int32_t n, int32_t elem_bytes, const void* w, void* u,
                                 double* scratch, void* stream) {
  using namespace maxe;
  if (n < 0 || (elem_bytes != 4 && elem_bytes != 8) || (n > 0 && (!w || !u || !scratch))) return MAXE_ERR_INVALID;
  if (n == 0) return MAXE_OK;
  cudaStream_t st = as_stream(stream);
  if (elem_bytes == 8)
    return norm_gather(Q, n, static_cast<const double*>(w), static_cast<double*>(u), scratch, st);
  return norm_gather(Q, n, static_cast<const float*>(w), static_cast<float*>(u), scratch, st);
}

maxe_status maxe_vec_dot_gather(const int32_t* Q, int32_t n, int32_t elem_bytes, const void* u, const void* w,
                                double* scratch, double* out, void* stream) {
  using namespace maxe;
  if (n < 0 || (elem_bytes != 4 && elem_bytes != 8) || !out || (n > 0 && (!w || !u || !scratch)))
    return MAXE_ERR_INVALID;
  cudaStream_t st = as_stream(stream);
  if (n == 0) {
    MAXE_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), st));
    return MAXE_OK;
  }
  if (elem_bytes == 8)
    return dot_gather(Q, n, static_cast<const double*>(u), static_cast<const double*>(w), scratch, out, st);
  return dot_gather(Q, n, static_cast<const float*>(u), static_cast<const float*>(w), scratch, out, st);
}

}  // extern "C"
