// k_factor_cluster.cu -- the element-block factorisation of k_blocks.cu
// (Section 2.4: the smoother's blocks D_e, power-of-two equilibration, then
// Gauss-Jordan elimination with partial pivoting to the explicit inverse) for
// blocks too large for one CTA's shared memory: hexahedra at P = 3 have
// n = 5 (P+1)^3 = 320, 400 KB in FP32.
//
// A thread-block cluster of C CTAs (2, 4 or 8) owns one block.  CTA r keeps
// columns [r nc, (r+1) nc) of the equilibrated matrix in its shared memory
// (nc = ceil(n / C)); every step k of the elimination needs from the rest of
// the cluster only the pivot row index and the pivot column, which the CTA
// owning column k publishes in its shared memory and the others read through
// distributed shared memory, between two cluster barriers.  Row interchanges
// and the updates of each CTA's columns are local.  The operations on every
// entry are those of the one-CTA kernel in the same order, so both give the
// same inverse bit for bit.  The final column interchanges (the row
// interchanges undone) become a permutation of the stored columns.
#include <cooperative_groups.h>

#include "pmg_internal.h"

namespace cg = cooperative_groups;

namespace pmg {

namespace {

__device__ __forceinline__ double pow2_inv_scale_c(double m) {
  // 2^-k with m * 2^-k in [0.5, 1); 1 for m == 0 (as in the one-CTA kernel)
  if (!(m > 0.0)) return 1.0;
  int ex;
  frexp(m, &ex);
  return ldexp(1.0, -ex);
}

template <class W> struct EpsC;
template <> struct EpsC<float> { static constexpr double value = 1.1920928955078125e-07; };
template <> struct EpsC<double> { static constexpr double value = 2.220446049250313e-16; };

}  // namespace

// One CTA per SM (its shared memory fills it): 1024 threads keep enough warps
// in flight for the elimination's shared-memory round trips.
constexpr int kClusterThreads = 1024;

// Shared memory of one CTA: doubles (row maxima, row scales, own column
// scales), then the acc-type arrays (own columns, column k, published column
// k), then ints (interchanges, column order, its inverse).
size_t factor_cluster_smem(int n, int C, int tbytes) {
  const size_t nc = (size_t)(n + C - 1) / C;
  return 8 * (2 * (size_t)n + nc) + (size_t)tbytes * ((size_t)n * nc + 2 * (size_t)n) + 4 * (3 * (size_t)n);
}

template <class W, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kClusterThreads)
    factor_cluster_kernel(int n, const double* __restrict__ Din, W* __restrict__ Dinv, double* __restrict__ rs,
                          double* __restrict__ cs, int* __restrict__ flag, int flag_base) {
  using T = typename Blk<W>::acc;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int e = blockIdx.x / C;
  const int nc = (n + C - 1) / C;
  const int c0 = rank * nc, c1 = min(n, c0 + nc), m = c1 > c0 ? c1 - c0 : 0;
  extern __shared__ __align__(16) unsigned char raw[];
  double* rowm = reinterpret_cast<double*>(raw);   // n: row maxima over own columns (published)
  double* sr = rowm + n;                            // n: row scales
  double* sc = sr + n;                              // nc: own column scales
  T* A = reinterpret_cast<T*>(sc + nc);             // n x nc, row-major
  T* colk = A + (size_t)n * nc;                     // n: column k (local copy)
  T* colpub = colk + n;                             // n: column k as published by its owner
  int* perm = reinterpret_cast<int*>(colpub + n);   // n: row interchanges
  int* idx = perm + n;                              // n: source column of each output column
  int* inv = idx + n;                               // n: output column of each source column
  __shared__ int s_piv, s_bad;
  __shared__ T s_ipiv;
  const double* D = Din + (size_t)e * n * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  // row scales from the maxima of every CTA's columns
  for (int i = tid; i < n; i += nt) {
    double mx = 0.0;
    for (int j = c0; j < c1; ++j) mx = fmax(mx, fabs(D[(size_t)i * n + j]));
    rowm[i] = mx;
  }
  cl.sync();
  for (int i = tid; i < n; i += nt) {
    double mx = 0.0;
    for (int r = 0; r < C; ++r) mx = fmax(mx, cl.map_shared_rank(rowm, r)[i]);
    sr[i] = pow2_inv_scale_c(mx);
  }
  __syncthreads();
  for (int jl = tid; jl < m; jl += nt) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(D[(size_t)i * n + c0 + jl] * sr[i]));
    sc[jl] = pow2_inv_scale_c(mx);
  }
  __syncthreads();
  for (int t = tid; t < n * m; t += nt) {
    const int i = t / m, jl = t - i * m;
    A[(size_t)i * nc + jl] = (T)(D[(size_t)i * n + c0 + jl] * sr[i] * sc[jl]);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int owner = k / nc, kl = k - owner * nc;
    if (rank == owner && tid < 32) {   // partial pivoting in the owner's column k
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < n; i += 32) {
        const double a = fabs((double)A[(size_t)i * nc + kl]);
        if (a > best) { best = a; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        if (!(best > n * EpsC<T>::value) || isinf(best)) s_bad = 1;
      }
    }
    cl.sync();
    const int p = *cl.map_shared_rank(&s_piv, owner);
    if (tid == 0) perm[k] = p;
    if (p != k)
      for (int jl = tid; jl < m; jl += nt) {
        const T t = A[(size_t)k * nc + jl];
        A[(size_t)k * nc + jl] = A[(size_t)p * nc + jl];
        A[(size_t)p * nc + jl] = t;
      }
    __syncthreads();
    if (rank == owner) {
      if (tid == 0) s_ipiv = (T)1 / A[(size_t)k * nc + kl];
      for (int i = tid; i < n; i += nt) colpub[i] = A[(size_t)i * nc + kl];
    }
    cl.sync();
    const T ipiv = *cl.map_shared_rank(&s_ipiv, owner);
    const T* pub = cl.map_shared_rank(colpub, owner);
    for (int i = tid; i < n; i += nt) colk[i] = pub[i];
    for (int jl = tid; jl < m; jl += nt)
      A[(size_t)k * nc + jl] = (c0 + jl == k) ? ipiv : A[(size_t)k * nc + jl] * ipiv;
    __syncthreads();
    // The update of the own columns; every entry sees the same operation as
    // in the one-CTA kernel.  FP32 elimination (issue-bound): thread (r0, jl)
    // updates column jl in rows r0, r0 + rpp, ... (rpp = nt / m rows per
    // pass), the pivot row's entry in a register and no index divided in the
    // loop -- 1.57x faster on n = 320.  FP64 elimination (bound by the FP64
    // pipe): all threads over the flattened n x m entries, which balances the
    // FP64 work exactly.
    if (sizeof(T) == 4) {
      if (m > 0) {
        const int rpp = nt / m, jl = tid % m, r0 = tid / m;
        if (r0 < rpp) {
          const T akj = A[(size_t)k * nc + jl];
          const bool kcol = c0 + jl == k;
          for (int i = r0; i < n; i += rpp) {
            if (i == k) continue;
            const T f = colk[i];
            if (kcol) A[(size_t)i * nc + jl] = -f * akj;
            else A[(size_t)i * nc + jl] -= f * akj;
          }
        }
      }
    } else {
      for (int t = tid; t < n * m; t += nt) {
        const int i = t / m, jl = t - i * m;
        if (i == k) continue;
        const T f = colk[i];
        if (c0 + jl == k) A[(size_t)i * nc + jl] = -f * A[(size_t)k * nc + jl];
        else A[(size_t)i * nc + jl] -= f * A[(size_t)k * nc + jl];
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first: as a
  // permutation of the columns
  if (tid == 0) {
    for (int j = 0; j < n; ++j) idx[j] = j;
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      const int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
    for (int j = 0; j < n; ++j) inv[idx[j]] = j;
  }
  __syncthreads();
  // store column-major: Dinv[e][col][row]
  W* out = Dinv + (size_t)e * n * n;
  for (int t = tid; t < m * n; t += nt) {
    const int jl = t / n, row = t - jl * n;
    out[(size_t)inv[c0 + jl] * n + row] = (W)A[(size_t)row * nc + jl];
  }
  if (rank == 0)
    for (int i = tid; i < n; i += nt) rs[(size_t)e * n + i] = sr[i];
  for (int jl = tid; jl < m; jl += nt) cs[(size_t)e * n + c0 + jl] = sc[jl];
  if (tid == 0 && s_bad) atomicMax(flag, flag_base + e + 1);
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

namespace {

size_t one_cta_smem(int n, int tbytes) {   // the k_blocks.cu kernel's layout
  size_t b = (size_t)n * n * tbytes + (size_t)n * tbytes + (size_t)n * 4;
  b = (b + 7) & ~(size_t)7;
  return b + 2 * (size_t)n * 8;
}

constexpr size_t kSmemBudget = (size_t)227 * 1024 - 64;   // dynamic bytes a CTA may take

template <class W>
void launch_cluster_w(int C, int n, int E, const double* D, W* Dinv, double* rs, double* cs, int* flag, int base,
                      cudaStream_t s) {
  const size_t bytes = factor_cluster_smem(n, C, (int)sizeof(typename Blk<W>::acc));
  if (C == 2) factor_cluster_kernel<W, 2><<<E * 2, kClusterThreads, bytes, s>>>(n, D, Dinv, rs, cs, flag, base);
  else if (C == 4) factor_cluster_kernel<W, 4><<<E * 4, kClusterThreads, bytes, s>>>(n, D, Dinv, rs, cs, flag, base);
  else factor_cluster_kernel<W, 8><<<E * 8, kClusterThreads, bytes, s>>>(n, D, Dinv, rs, cs, flag, base);
}

template <class W>
cudaError_t prepare_w(int C, size_t bytes) {
  if (C == 2) return cudaFuncSetAttribute(factor_cluster_kernel<W, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (C == 4) return cudaFuncSetAttribute(factor_cluster_kernel<W, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(factor_cluster_kernel<W, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// CTAs per block: 1 (the one-CTA kernel of k_blocks.cu), 2, 4 or 8 (a
// cluster), 0 when even 8 CTAs cannot hold it.  PMG_FACTOR_CLUSTER = 2, 4 or 8
// puts every block that such a cluster holds on the cluster kernel (tests).
int factor_cluster_size(int n, int prec) {
  const int tb = prec == PMG_PREC_FP64 ? 8 : 4;
  int force = 0;
  if (const char* env = getenv("PMG_FACTOR_CLUSTER")) force = atoi(env);
  if ((force == 2 || force == 4 || force == 8) && factor_cluster_smem(n, force, tb) <= kSmemBudget) return force;
  if (one_cta_smem(n, tb) <= (size_t)227 * 1024) return 1;
  for (int C : {2, 4, 8})
    if (factor_cluster_smem(n, C, tb) <= kSmemBudget) return C;
  return 0;
}

void launch_factor_cluster(const Ctx& c, LevelDev& L, int level, int prec, int C, int* flag, cudaStream_t s) {
  const int base = level * c.E;
  if (prec == PMG_PREC_FP64)
    launch_cluster_w<double>(C, L.n, c.E, L.Dfull, (double*)L.Dinv, L.rs, L.cs, flag, base, s);
  else if (prec == PMG_PREC_BF16R)
    launch_cluster_w<__nv_bfloat16>(C, L.n, c.E, L.Dfull, (__nv_bfloat16*)L.Dinv, L.rs, L.cs, flag, base, s);
  else
    launch_cluster_w<float>(C, L.n, c.E, L.Dfull, (float*)L.Dinv, L.rs, L.cs, flag, base, s);
}

cudaError_t prepare_factor_cluster(int n, int prec, int C) {
  const size_t bytes = factor_cluster_smem(n, C, prec == PMG_PREC_FP64 ? 8 : 4);
  if (prec == PMG_PREC_FP64) return prepare_w<double>(C, bytes);
  if (prec == PMG_PREC_BF16R) return prepare_w<__nv_bfloat16>(C, bytes);
  return prepare_w<float>(C, bytes);
}

}  // namespace pmg
