// k_krylov.cu -- vector kernels of the Newton-Krylov stage solver (api.cu
// nk_stage_solve): several inner products in one launch (the classical
// Gram-Schmidt steps of FGMRES), y += sign sum_j c_j X_j, and linear
// combinations whose terms carry a scale per state variable (the vectors are
// SoA planes of E N values per variable).  All of it is HBM-bound streaming
// over the finest level's vectors.
#include "pmg_internal.h"

namespace pmg {

constexpr int kKrylovThreads = 256;
constexpr int kMaxCombine = 64;

__device__ __forceinline__ double block_sum(double s, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;   // valid in thread 0
}

// Block (x, j): partial sum of X_j . y over a grid-stride range of indices.
__global__ void __launch_bounds__(kKrylovThreads) multi_dot_partial_kernel(const double* __restrict__ X, size_t ld,
                                                                          const double* __restrict__ y, size_t n,
                                                                          double* __restrict__ part) {
  __shared__ double sm[kKrylovThreads / 32];
  const double* x = X + (size_t)blockIdx.y * ld;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s, sm);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Block j: the kDotBlocks partial sums of product j, in a fixed order.
__global__ void __launch_bounds__(kKrylovThreads) sum_partials_kernel(const double* __restrict__ part, int nb,
                                                                     double* __restrict__ out) {
  __shared__ double sm[kKrylovThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(size_t)blockIdx.x * nb + i];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

void launch_multi_dot(const double* X, size_t ld, int k, const double* y, size_t n, double* part, double* out,
                      cudaStream_t s) {
  if (k <= 0) return;
  multi_dot_partial_kernel<<<dim3(kDotBlocks, k), kKrylovThreads, 0, s>>>(X, ld, y, n, part);
  sum_partials_kernel<<<k, kKrylovThreads, 0, s>>>(part, kDotBlocks, out);
}

__global__ void __launch_bounds__(kKrylovThreads) combination_kernel(double* __restrict__ y,
                                                                    const double* __restrict__ X, size_t ld, int k,
                                                                    const double* __restrict__ coef, double sign,
                                                                    size_t n) {
  __shared__ double c[kMaxCombine];
  if (threadIdx.x < k) c[threadIdx.x] = sign * coef[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(c[j], X[(size_t)j * ld + i], acc);
    y[i] += acc;
  }
}

void launch_combination(double* y, const double* X, size_t ld, int k, const double* coef, double sign, size_t n,
                        cudaStream_t s) {
  if (k <= 0) return;
  const size_t want = (n + kKrylovThreads - 1) / kKrylovThreads;
  const unsigned blocks = (unsigned)(want < (size_t)4 * kDotBlocks ? want : (size_t)4 * kDotBlocks);
  combination_kernel<<<blocks, kKrylovThreads, 0, s>>>(y, X, ld, k < kMaxCombine ? k : kMaxCombine, coef, sign, n);
}

__global__ void __launch_bounds__(kKrylovThreads) plane_combine_kernel(double* out, const double* x0, double a0,
                                                                      const double* x1, double a1, Scale5 s0,
                                                                      const double* x2, double a2, Scale5 s2,
                                                                      size_t plane, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(i / plane);
    double t = 0.0;
    if (x0) t = a0 * x0[i];
    if (x1) t = fma(a1, x1[i], t);
    t *= s0.s[v];
    if (x2) t = fma(a2 * s2.s[v], x2[i], t);
    out[i] = t;
  }
}

void launch_plane_combine(double* out, const double* x0, double a0, const double* x1, double a1, const Scale5& s0,
                          const double* x2, double a2, const Scale5& s2, size_t plane, size_t n, cudaStream_t s) {
  const size_t want = (n + kKrylovThreads - 1) / kKrylovThreads;
  const unsigned blocks = (unsigned)(want < (size_t)4 * kDotBlocks ? want : (size_t)4 * kDotBlocks);
  plane_combine_kernel<<<blocks, kKrylovThreads, 0, s>>>(out, x0, a0, x1, a1, s0, x2, a2, s2, plane, n);
}

}  // namespace pmg
