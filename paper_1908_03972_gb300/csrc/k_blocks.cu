// k_blocks.cu -- element-Jacobi smoother blocks (Section 2.4, eqs.
// linearized_pseudo_transient_final and smoothing_element_jacobi).
//
//  * assemble: one CTA per element builds D_e = Gamma/dtau + M/(omega dt)
//    - dR_e/dq_e in FP64.  dR_e/dq_e is exact: pointwise flux Jacobians and
//    the own-side derivative of the preconditioned Roe flux (including its
//    dependence through the averaged state) come from forward-mode dual
//    numbers pushed through the same flux code as the residual; the FR
//    structure (derivative, extrapolation, correction) is applied in
//    tensor-product form.  Neighbour states are frozen.
//  * factor: one CTA per element equilibrates the block with power-of-two
//    row and column scales (exact in any precision) and inverts it by
//    Gauss-Jordan elimination with partial pivoting in the working precision
//    (FP64, or FP32 for the mixed-precision smoother).  The explicit inverse
//    turns every smoothing sweep into a batched matrix-vector product.  The
//    equilibrated rows have unit size, so a pivot that is not finite or not
//    above n eps of the working precision (the rounding a dependent row leaves
//    after elimination) marks a block that is singular to that precision: the
//    element is flagged for the host (PMG_ESINGULAR).
//  * apply: x = cs .* (inv(D^) (rs .* r)); each thread owns four consecutive
//    rows and streams the column-major inverse with 16-byte (FP32) or
//    2x16-byte (FP64) loads.  This stream is the smoother's HBM/L2 traffic.
#include <cstdint>
#include <algorithm>

#include "pmg_internal.h"

namespace pmg {

// ------------------------------------------------------------------ assemble
template <int P>
__global__ void __launch_bounds__(128) assemble_kernel(int E, const double* __restrict__ q,
                                                       const double* __restrict__ met,
                                                       const double* __restrict__ face,
                                                       const int* __restrict__ nbr, OpTab op, Phys ph,
                                                       const double* __restrict__ d_dtau, double inv_odt,
                                                       double* __restrict__ Dout) {
  constexpr int n1 = P + 1, N = n1 * n1, n = 4 * N;
  __shared__ double sq[4][N];
  __shared__ double sAx[N][16], sAe[N][16], sDiag[N][16];
  __shared__ double sC[4][n1][16];
  __shared__ double sinvJ[N];
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  const int e = blockIdx.x;
  const size_t plane = (size_t)E * N;
  const double dtau = *d_dtau;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) sq[t / N][t % N] = q[(t / N) * plane + (size_t)e * N + t % N];
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = op.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = op.gL[threadIdx.x];
    sgR[threadIdx.x] = op.gR[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  __syncthreads();
  // pointwise contravariant flux Jacobians and the pseudo/physical time terms
  for (int pt = threadIdx.x; pt < N; pt += blockDim.x) {
    size_t gi = (size_t)e * N + pt;
    double a = met[gi], b = met[plane + gi], c = met[2 * plane + gi], d = met[3 * plane + gi];
    sinvJ[pt] = met[4 * plane + gi];
    double qv[4] = {sq[0][pt] + ph.p_ref, sq[1][pt], sq[2][pt], sq[3][pt]};   // absolute pressure
    for (int w = 0; w < 4; ++w) {
      Dual qd[4];
      for (int k = 0; k < 4; ++k) qd[k] = Dual(qv[k], k == w ? 1.0 : 0.0);
      Dual f[4], g[4];
      flux_xy(qd, qd[0] - ph.p_ref, ph, f, g);
      for (int v = 0; v < 4; ++v) {
        sAx[pt][v * 4 + w] = a * f[v].d + b * g[v].d;
        sAe[pt][v * 4 + w] = c * f[v].d + d * g[v].d;
      }
    }
    double G[16], M[16];
    gamma_and_M(qv, ph, G, M);
    for (int i = 0; i < 16; ++i) sDiag[pt][i] = G[i] / dtau + M[i] * inv_odt;
  }
  // own-side derivative of the reference-direction common flux at each face point
  for (int t = threadIdx.x; t < 4 * n1; t += blockDim.x) {
    int f = t / n1, k = t - f * n1;
    const bool plus = (f == 1 || f == 2);
    const bool eta = (f == 0 || f == 2);
    double qm[4], qp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int v = 0; v < 4; ++v) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) s += (plus ? slp[m] : slm[m]) * sq[v][eta ? m * n1 + k : k * n1 + m];
      qm[v] = s;
    }
    int en = nbr[(e * 4 + f) * 3 + 0], fn = nbr[(e * 4 + f) * 3 + 1], rev = nbr[(e * 4 + f) * 3 + 2];
    int kn = rev ? P - k : k;
    if (en >= 0) {
      const bool pn = (fn == 1 || fn == 2);
      const bool en_eta = (fn == 0 || fn == 2);
      for (int v = 0; v < 4; ++v) {
        double s = 0.0;
        for (int m = 0; m < n1; ++m)
          s += (pn ? slp[m] : slm[m]) * q[v * plane + (size_t)en * N + (en_eta ? m * n1 + kn : kn * n1 + m)];
        qp[v] = s;
      }
      qp[0] += ph.p_ref;
    }
    qm[0] += ph.p_ref;
    const double* g = face + (((size_t)e * 4 + f) * n1 + k) * 3;
    double sg = plus ? 1.0 : -1.0;
    for (int w = 0; w < 4; ++w) {
      Dual dm[4], dp[4], o[4];
      for (int v = 0; v < 4; ++v) { dm[v] = Dual(qm[v], v == w ? 1.0 : 0.0); dp[v] = Dual(qp[v], 0.0); }
      // a boundary face's ghost state follows the own trace (fn = boundary type)
      if (en < 0) ghost_state(fn, dm, g[0], g[1], ph, dp);
      roe_flux(dm, dp, g[0], g[1], g[2], ph, o);
      for (int v = 0; v < 4; ++v) sC[f][k][v * 4 + w] = sg * o[v].d;
    }
  }
  __syncthreads();
  // fill the block: D = diag terms - dR/dq, with dR/dq = -(1/|J|) d(div + corr)/dq
  double* Db = Dout + (size_t)e * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int row = t / n, col = t - row * n;
    int v = row / N, rp = row - v * N, w = col / N, cp = col - w * N;
    int i = rp % n1, j = rp / n1, k = cp % n1, l = cp / n1;
    int vw = v * 4 + w;
    double s = 0.0;
    if (l == j) {   // same xi line
      double A = sAx[cp][vw];
      s += sD[i][k] * A;
      s += sgL[i] * slm[k] * (sC[3][j][vw] - A);
      s += sgR[i] * slp[k] * (sC[1][j][vw] - A);
    }
    if (k == i) {   // same eta line
      double A = sAe[cp][vw];
      s += sD[j][l] * A;
      s += sgL[j] * slm[l] * (sC[0][i][vw] - A);
      s += sgR[j] * slp[l] * (sC[2][i][vw] - A);
    }
    double val = s * sinvJ[rp];
    if (rp == cp) val += sDiag[rp][vw];
    Db[t] = val;
  }
}

void launch_assemble(const Ctx& c, const LevelDev& L, const double* q, const double* d_dtau, double inv_odt,
                     cudaStream_t s) {
  if (c.dim == 3) { launch_assemble3(c, L, q, d_dtau, inv_odt, s); return; }
  const int* nbr = c.d_faces + 5 * c.n_faces;   // neighbour table stored after the face list
#define PMG_ASM(PP) \
  assemble_kernel<PP><<<c.E, 128, 0, s>>>(c.E, q, L.met, L.face, nbr, L.op, c.ph, d_dtau, inv_odt, L.Dfull)
  switch (L.P) {
    case 0: PMG_ASM(0); break;
    case 1: PMG_ASM(1); break;
    case 2: PMG_ASM(2); break;
    case 3: PMG_ASM(3); break;
    case 4: PMG_ASM(4); break;
    default: PMG_ASM(5); break;
  }
#undef PMG_ASM
  if (c.ph.mu > 0.0) launch_assemble_visc(c, L, q, s);
}

// -------------------------------------------------------------------- factor
__device__ __forceinline__ double pow2_inv_scale(double m) {
  // 2^-k with m * 2^-k in [0.5, 1); 1 for m == 0
  if (!(m > 0.0)) return 1.0;
  int ex;
  frexp(m, &ex);
  return ldexp(1.0, -ex);
}

// Machine epsilon of the working precision; the smallest pivot magnitude
// accepted is n eps (the equilibrated rows have unit size).
template <class W> struct Eps;
template <> struct Eps<float> { static constexpr double value = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double value = 2.220446049250313e-16; };

template <class W>
__global__ void __launch_bounds__(256) factor_kernel(int n, const double* __restrict__ Din, W* __restrict__ Dinv,
                                                     double* __restrict__ rs, double* __restrict__ cs,
                                                     int* __restrict__ flag, int flag_base) {
  using T = typename Blk<W>::acc;   // elimination arithmetic (FP32 for BF16 storage)
  extern __shared__ unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);                       // n * n, row-major
  T* colk = A + n * n;                                          // n
  int* perm = reinterpret_cast<int*>(colk + n);                 // n
  double* sr = reinterpret_cast<double*>(((uintptr_t)(perm + n) + 7) & ~(uintptr_t)7);   // n
  double* sc = sr + n;                                          // n
  __shared__ int s_piv;
  __shared__ int s_bad;
  const int e = blockIdx.x;
  const double* D = Din + (size_t)e * n * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  // row scales
  for (int i = tid; i < n; i += nt) {
    double m = 0.0;
    for (int j = 0; j < n; ++j) m = fmax(m, fabs(D[(size_t)i * n + j]));
    sr[i] = pow2_inv_scale(m);
  }
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(D[(size_t)i * n + j] * sr[i]));
    sc[j] = pow2_inv_scale(m);
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) {
    int i = t / n, j = t - i * n;
    A[t] = (T)(D[t] * sr[i] * sc[j]);
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting, in place
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < n; i += 32) {
        double a = fabs((double)A[i * n + k]);
        if (a > best) { best = a; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (!(best > n * Eps<T>::value) || isinf(best)) s_bad = 1;
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k)
      for (int j = tid; j < n; j += nt) { T t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
    __syncthreads();
    T piv = A[k * n + k];
    T ipiv = (T)1 / piv;
    __syncthreads();
    for (int j = tid; j < n; j += nt) A[k * n + j] = (j == k) ? ipiv : A[k * n + j] * ipiv;
    for (int i = tid; i < n; i += nt) colk[i] = A[i * n + k];
    __syncthreads();
    if (sizeof(T) == 4 && n <= nt) {
      // FP32 elimination (issue-bound): thread (r0, j) updates column j in
      // rows r0, r0 + rpp, ... with the pivot row's entry in a register and
      // no index division; the same operation on every entry as below
      const int rpp = nt / n, j = tid % n, r0 = tid / n;
      if (r0 < rpp) {
        const T akj = A[k * n + j];
        for (int i = r0; i < n; i += rpp) {
          if (i == k) continue;
          const T f = colk[i];
          if (j == k) A[i * n + j] = -f * akj;
          else A[i * n + j] -= f * akj;
        }
      }
    } else {
      for (int t = tid; t < n * n; t += nt) {
        int i = t / n, j = t - i * n;
        if (i == k) continue;
        T f = colk[i];
        if (j == k) A[t] = -f * A[k * n + k];
        else A[t] -= f * A[k * n + j];
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    int p = perm[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) { T t = A[i * n + k]; A[i * n + k] = A[i * n + p]; A[i * n + p] = t; }
    __syncthreads();
  }
  // store column-major: Dinv[e][col][row]
  W* out = Dinv + (size_t)e * n * n;
  for (int t = tid; t < n * n; t += nt) {
    int col = t / n, row = t - col * n;
    out[t] = (W)A[row * n + col];
  }
  for (int i = tid; i < n; i += nt) {
    rs[(size_t)e * n + i] = sr[i];
    cs[(size_t)e * n + i] = sc[i];
  }
  if (tid == 0 && s_bad) atomicMax(flag, flag_base + e + 1);
}

static size_t factor_smem(int n, int wbytes) {
  size_t b = (size_t)n * n * wbytes + (size_t)n * wbytes + (size_t)n * 4;
  b = (b + 7) & ~(size_t)7;
  return b + 2 * (size_t)n * 8;
}

void launch_factor(const Ctx& c, LevelDev& L, int level, int prec, int* flag, cudaStream_t s) {
  const int n = L.n, base = level * c.E;   // the flag holds 1 + level E + element of the highest bad block
  const int C = factor_cluster_size(n, prec);
  if (C > 1) {   // too large for one CTA: a cluster of C (k_factor_cluster.cu)
    launch_factor_cluster(c, L, level, prec, C, flag, s);
    return;
  }
  if (prec == PMG_PREC_FP64)
    factor_kernel<double><<<c.E, 256, factor_smem(n, 8), s>>>(n, L.Dfull, (double*)L.Dinv, L.rs, L.cs, flag, base);
  else if (prec == PMG_PREC_BF16R)
    factor_kernel<__nv_bfloat16><<<c.E, 256, factor_smem(n, 4), s>>>(n, L.Dfull, (__nv_bfloat16*)L.Dinv, L.rs,
                                                                       L.cs, flag, base);
  else
    factor_kernel<float><<<c.E, 256, factor_smem(n, 4), s>>>(n, L.Dfull, (float*)L.Dinv, L.rs, L.cs, flag, base);
}

// Largest block the shared-memory factorisation holds in the precision prec:
// one CTA (227 KB) up to n = 168 in FP64 and 238 in FP32 and BF16 (their
// elimination runs in FP32), a cluster of up to 8 CTAs beyond.
int factor_max_n(int prec) {
  int n = 4;
  while (factor_cluster_size(n + 1, prec) > 0) ++n;
  return n;
}

// Opt the factor kernels into the dynamic shared memory the largest block
// needs (done once, outside any stream capture).  Levels whose blocks exceed
// factor_max_n are left out; the calls that would factor them fail first.
cudaError_t prepare_kernels(const Ctx& c) {
  int nmax = 4;
  for (int l = 0; l < c.cfg.n_levels; ++l) {
    const int C = factor_cluster_size(c.lev[l].n, c.cfg.block_prec);
    if (C == 1) nmax = std::max(nmax, c.lev[l].n);
    if (C > 1) {
      cudaError_t e = prepare_factor_cluster(c.lev[l].n, c.cfg.block_prec, C);
      if (e != cudaSuccess) return e;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)factor_smem(nmax, 8));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(factor_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)factor_smem(nmax, 4));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(factor_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)factor_smem(nmax, 4));
}

// --------------------------------------------------------------------- apply
template <class W> struct Vec4;
template <> struct Vec4<float> {
  __device__ static inline void load(const float* p, float o[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
};
template <> struct Vec4<__nv_bfloat16> {
  __device__ static inline void load(const __nv_bfloat16* p, float o[4]) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    o[0] = lo.x; o[1] = lo.y; o[2] = hi.x; o[3] = hi.y;
  }
};
template <> struct Vec4<double> {
  __device__ static inline void load(const double* p, double o[4]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
};

// One thread per four rows of one element's block; N threads per element.
template <int N>
struct ApplyEPB {   // elements per CTA: 1-2 warps per CTA, enough CTAs for all SMs
  static constexpr int value = N <= 4 ? 32 / N : (64 / N > 0 ? 64 / N : 1);
};

template <class W, int N>
__global__ void __launch_bounds__(64) apply_kernel(int E, const W* __restrict__ Dinv, const double* __restrict__ rs,
                                                   const double* __restrict__ cs, const double* __restrict__ r,
                                                   double* __restrict__ x, int accumulate) {
  constexpr int n = 4 * N;
  constexpr int EPB = ApplyEPB<N>::value;
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[EPB][n];
  const int le = threadIdx.x / N, t = threadIdx.x - le * N;
  const int e = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (e < E);
  const size_t plane = (size_t)E * N;
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int row = v * N + t;
      sr[le][row] = scaled_in<W>(r[v * plane + (size_t)e * N + t], rs[(size_t)e * n + row]);
    }
  }
  __syncthreads();
  if (!active) return;
  Acc acc[4] = {0, 0, 0, 0};
  const W* Dm = Dinv + (size_t)e * n * n + 4 * t;
#pragma unroll 8
  for (int k = 0; k < n; ++k) {
    Acc d[4];
    Vec4<W>::load(Dm + (size_t)k * n, d);
    Acc rk = sr[le][k];
    acc[0] = fma(d[0], rk, acc[0]);
    acc[1] = fma(d[1], rk, acc[1]);
    acc[2] = fma(d[2], rk, acc[2]);
    acc[3] = fma(d[3], rk, acc[3]);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int row = 4 * t + m;
    int v = row / N, pt = row - v * N;
    double xv = scaled_out<W>(acc[m], cs[(size_t)e * n + row]);
    size_t o = v * plane + (size_t)e * N + pt;
    if (accumulate) x[o] += xv;
    else x[o] = xv;
  }
}

template <class W>
static void apply_dispatch(const Ctx& c, const LevelDev& L, const W* Dinv, const double* r, double* x, int acc,
                           cudaStream_t s) {
  int N = L.N;
  int epb = 1;
  switch (N) {
    case 1: epb = ApplyEPB<1>::value; break;
    case 4: epb = ApplyEPB<4>::value; break;
    case 9: epb = ApplyEPB<9>::value; break;
    case 16: epb = ApplyEPB<16>::value; break;
    case 25: epb = ApplyEPB<25>::value; break;
    default: epb = ApplyEPB<36>::value; break;
  }
  int threads = ((epb * N) + 31) / 32 * 32;
  int blocks = (c.E + epb - 1) / epb;
#define PMG_APPLY(NN) apply_kernel<W, NN><<<blocks, threads, 0, s>>>(c.E, Dinv, L.rs, L.cs, r, x, acc)
  switch (N) {
    case 1: PMG_APPLY(1); break;
    case 4: PMG_APPLY(4); break;
    case 9: PMG_APPLY(9); break;
    case 16: PMG_APPLY(16); break;
    case 25: PMG_APPLY(25); break;
    default: PMG_APPLY(36); break;
  }
#undef PMG_APPLY
}

void launch_apply(const Ctx& c, const LevelDev& L, int prec, const double* r, double* x, int accumulate,
                  cudaStream_t s) {
  if (c.dim == 3) { launch_apply3(c, L, prec, r, x, accumulate, s); return; }
  if (prec == PMG_PREC_FP64) apply_dispatch<double>(c, L, (const double*)L.Dinv, r, x, accumulate, s);
  else if (prec == PMG_PREC_BF16R)
    apply_dispatch<__nv_bfloat16>(c, L, (const __nv_bfloat16*)L.Dinv, r, x, accumulate, s);
  else apply_dispatch<float>(c, L, (const float*)L.Dinv, r, x, accumulate, s);
}

}  // namespace pmg
