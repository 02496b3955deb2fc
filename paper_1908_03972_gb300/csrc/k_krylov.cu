// k_krylov.cu -- vector kernels of the Newton-Krylov stage solver (api.cu
// nk_stage_solve): several inner products in one launch (the classical
// Gram-Schmidt steps of FGMRES), y += sign sum_j c_j X_j, and linear
// combinations whose terms carry a scale per state variable (the vectors are
// SoA planes of E N values per variable).  All of it is HBM-bound streaming
// over the finest level's vectors.
#include "physics3.cuh"
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

// Largest relative change |dx| / |x (+ p_ref for the pressure)| over the
// pressure plane (v = 0) and the temperature plane (v = tslot); a non-finite
// ratio counts as 1e300.  One partial maximum per block, then one block.
__device__ __forceinline__ double block_max(double m, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  return m;
}

__global__ void __launch_bounds__(kKrylovThreads) rel_change_partial_kernel(const double* __restrict__ x,
                                                                           const double* __restrict__ dx,
                                                                           size_t plane, int tslot, double p_ref,
                                                                           double* __restrict__ part) {
  __shared__ double sm[kKrylovThreads / 32];
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * plane; i += (size_t)gridDim.x * blockDim.x) {
    const bool pres = i < plane;
    const size_t j = pres ? i : (size_t)tslot * plane + (i - plane);
    const double r = fabs(dx[j]) / fabs(pres ? x[j] + p_ref : x[j]);
    m = r <= 1e300 ? fmax(m, r) : 1e300;
  }
  m = block_max(m, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void __launch_bounds__(kKrylovThreads) max_partials_kernel(const double* __restrict__ part, int nb,
                                                                     double* __restrict__ out) {
  __shared__ double sm[kKrylovThreads / 32];
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, part[i]);
  m = block_max(m, sm);
  if (threadIdx.x == 0) out[0] = m;
}

void launch_rel_change(const double* x, const double* dx, size_t plane, int tslot, double p_ref, double* part,
                       double* out, cudaStream_t s) {
  rel_change_partial_kernel<<<kDotBlocks, kKrylovThreads, 0, s>>>(x, dx, plane, tslot, p_ref, part);
  max_partials_kernel<<<1, kKrylovThreads, 0, s>>>(part, kDotBlocks, out);
}

// out += a w_v (Gamma(q) z)_v at every point: the pseudo-time matrix of eq.
// preconditioning at the stored state q (pressure p - p_ref), applied to z.
__global__ void __launch_bounds__(kKrylovThreads) gamma_apply_kernel(int nv, size_t plane, const double* __restrict__ q,
                                                                    const double* __restrict__ z, double* out,
                                                                    double a, Scale5 w, Phys ph) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    if (nv == 4) {
      const double qv[4] = {q[i] + ph.p_ref, q[plane + i], q[2 * plane + i], q[3 * plane + i]};
      double G[16], M[16];
      gamma_and_M(qv, ph, G, M);
      for (int v = 0; v < 4; ++v) {
        double t = 0.0;
        for (int k = 0; k < 4; ++k) t = fma(G[v * 4 + k], z[k * plane + i], t);
        out[v * plane + i] += a * w.s[v] * t;
      }
    } else {
      const double qv[5] = {q[i] + ph.p_ref, q[plane + i], q[2 * plane + i], q[3 * plane + i], q[4 * plane + i]};
      double G[25], M[25];
      gamma_and_M3(qv, ph, G, M);
      for (int v = 0; v < 5; ++v) {
        double t = 0.0;
        for (int k = 0; k < 5; ++k) t = fma(G[v * 5 + k], z[k * plane + i], t);
        out[v * plane + i] += a * w.s[v] * t;
      }
    }
  }
}

void launch_gamma_apply(int nv, size_t plane, const double* q, const double* z, double* out, double a,
                        const Scale5& w, const Phys& ph, cudaStream_t s) {
  const size_t want = (plane + kKrylovThreads - 1) / kKrylovThreads;
  const unsigned blocks = (unsigned)(want < (size_t)4 * kDotBlocks ? want : (size_t)4 * kDotBlocks);
  gamma_apply_kernel<<<blocks, kKrylovThreads, 0, s>>>(nv, plane, q, z, out, a, w, ph);
}

}  // namespace pmg
