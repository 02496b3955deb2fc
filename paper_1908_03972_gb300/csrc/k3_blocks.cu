// k3_blocks.cu -- element-Jacobi blocks on hexahedra (Section 2.4, eqs.
// linearized_pseudo_transient_final and smoothing_element_jacobi, d = 3).
//
//  * assemble3: one CTA per element builds D_e = Gamma/dtau + M/(omega dt)
//    - dR_e/dq_e in FP64 (n = 5 (P+1)^3).  The pointwise Jacobians of the
//    contravariant fluxes and the own-side derivative of the common flux at
//    every face point (through the averaged state, and through the ghost
//    state on boundary faces) come from forward-mode dual numbers pushed
//    through the residual's flux code; the tensor-product FR structure
//    (derivative, extrapolation and correction along the three lines through
//    a point) fills the block.  Neighbours are frozen.
//  * apply3: x = cs .* (D^-1 (rs .* r)) with the factored inverse
//    (column-major); one thread per solution point forms its point's five
//    rows, so the threads of an element read every column contiguously.
// The factorisation is the dimension-independent factor kernel (k_blocks.cu).
#include "pmg_internal.h"
#include "physics3.cuh"

namespace pmg {

template <int P>
__global__ void __launch_bounds__(128) assemble3_kernel(int E, const double* __restrict__ q,
                                                        const double* __restrict__ met,
                                                        const double* __restrict__ face,
                                                        const int* __restrict__ nbr, OpTab op, Phys ph,
                                                        const double* __restrict__ d_dtau, double inv_odt,
                                                        double* __restrict__ Dout) {
  constexpr int n1 = P + 1, N = n1 * n1 * n1, NF = n1 * n1, n = 5 * N;
  extern __shared__ __align__(16) double dyn[];
  double* sA = dyn;                   // [N][3][25]: d(F^i)/dq_p at each point
  double* sC = sA + N * 75;           // [6][NF][25]: d(reference-direction common flux)/dq_p(own trace)
  double* sDiag = sC + 6 * NF * 25;   // [N][25]: Gamma/dtau + M/(omega dt)
  __shared__ double sq[5][N];
  __shared__ double sinvJ[N];
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  const int e = blockIdx.x;
  const size_t plane = (size_t)E * N;
  const double dtau = *d_dtau;
  for (int t = threadIdx.x; t < 5 * N; t += blockDim.x) sq[t / N][t % N] = q[(t / N) * plane + (size_t)e * N + t % N];
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = op.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = op.gL[threadIdx.x];
    sgR[threadIdx.x] = op.gR[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  __syncthreads();
  for (int pt = threadIdx.x; pt < N; pt += blockDim.x) {
    const size_t gi = (size_t)e * N + pt;
    sinvJ[pt] = met[9 * plane + gi];
    const double qv[5] = {sq[0][pt] + ph.p_ref, sq[1][pt], sq[2][pt], sq[3][pt], sq[4][pt]};
    for (int i = 0; i < 3; ++i) {
      const double ja[3] = {met[(3 * i) * plane + gi], met[(3 * i + 1) * plane + gi], met[(3 * i + 2) * plane + gi]};
      for (int w = 0; w < 5; ++w) {
        Dual qd[5];
        for (int c = 0; c < 5; ++c) qd[c] = Dual(qv[c], c == w ? 1.0 : 0.0);
        Dual f[5];
        flux3_n(qd, qd[0] - ph.p_ref, ja, ph, f);
        for (int v = 0; v < 5; ++v) sA[(pt * 3 + i) * 25 + v * 5 + w] = f[v].d;
      }
    }
    double G[25], M[25];
    gamma_and_M3(qv, ph, G, M);
    for (int c = 0; c < 25; ++c) sDiag[pt * 25 + c] = G[c] / dtau + M[c] * inv_odt;
  }
  for (int t = threadIdx.x; t < 6 * NF; t += blockDim.x) {
    const int f = t / NF, fp = t - f * NF, a = fp % n1, b = fp / n1, d = f >> 1;
    const bool plus = f & 1;
    double qm[5], qp[5] = {0, 0, 0, 0, 0};
    for (int v = 0; v < 5; ++v) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) {
        const int i = d == 0 ? m : a, j = d == 1 ? m : (d == 0 ? a : b), k = d == 2 ? m : b;
        s += (plus ? slp[m] : slm[m]) * sq[v][(k * n1 + j) * n1 + i];
      }
      qm[v] = s;
    }
    qm[0] += ph.p_ref;
    const int en = nbr[(e * 6 + f) * 3], fn = nbr[(e * 6 + f) * 3 + 1], o = nbr[(e * 6 + f) * 3 + 2];
    if (en >= 0) {
      const int s = (o & 4) ? b : a, tt = (o & 4) ? a : b;
      const int a2 = (o & 1) ? P - s : s, b2 = (o & 2) ? P - tt : tt;
      const int d2 = fn >> 1;
      const bool pn = fn & 1;
      for (int v = 0; v < 5; ++v) {
        double sum = 0.0;
        for (int m = 0; m < n1; ++m) {
          const int i = d2 == 0 ? m : a2, j = d2 == 1 ? m : (d2 == 0 ? a2 : b2), k = d2 == 2 ? m : b2;
          sum += (pn ? slp[m] : slm[m]) * q[v * plane + (size_t)en * N + (k * n1 + j) * n1 + i];
        }
        qp[v] = sum;
      }
      qp[0] += ph.p_ref;
    }
    const double* g = face + (((size_t)e * 6 + f) * NF + fp) * 4;
    const double nrm[3] = {g[0], g[1], g[2]};
    const double sg = plus ? 1.0 : -1.0;
    for (int w = 0; w < 5; ++w) {
      Dual dm[5], dp[5], out[5];
      for (int v = 0; v < 5; ++v) { dm[v] = Dual(qm[v], v == w ? 1.0 : 0.0); dp[v] = Dual(qp[v], 0.0); }
      if (en < 0) ghost_state3(fn, dm, nrm, ph, dp);   // a boundary face's ghost follows the own trace
      roe3_flux(dm, dp, nrm, g[3], ph, out);
      for (int v = 0; v < 5; ++v) sC[(f * NF + fp) * 25 + v * 5 + w] = sg * out[v].d;
    }
  }
  __syncthreads();
  double* Db = Dout + (size_t)e * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int row = t / n, col = t - row * n;
    const int v = row / N, rp = row - v * N, w = col / N, cp = col - w * N;
    const int i = rp % n1, j = (rp / n1) % n1, k = rp / NF;
    const int i2 = cp % n1, j2 = (cp / n1) % n1, k2 = cp / NF;
    const int vw = v * 5 + w;
    double s = 0.0;
    if (j2 == j && k2 == k) {   // xi line
      const double A = sA[(cp * 3 + 0) * 25 + vw];
      s += sD[i][i2] * A;
      s += sgL[i] * slm[i2] * (sC[(0 * NF + k * n1 + j) * 25 + vw] - A);
      s += sgR[i] * slp[i2] * (sC[(1 * NF + k * n1 + j) * 25 + vw] - A);
    }
    if (i2 == i && k2 == k) {   // eta line
      const double A = sA[(cp * 3 + 1) * 25 + vw];
      s += sD[j][j2] * A;
      s += sgL[j] * slm[j2] * (sC[(2 * NF + k * n1 + i) * 25 + vw] - A);
      s += sgR[j] * slp[j2] * (sC[(3 * NF + k * n1 + i) * 25 + vw] - A);
    }
    if (i2 == i && j2 == j) {   // zeta line
      const double A = sA[(cp * 3 + 2) * 25 + vw];
      s += sD[k][k2] * A;
      s += sgL[k] * slm[k2] * (sC[(4 * NF + j * n1 + i) * 25 + vw] - A);
      s += sgR[k] * slp[k2] * (sC[(5 * NF + j * n1 + i) * 25 + vw] - A);
    }
    double val = s * sinvJ[rp];
    if (rp == cp) val += sDiag[rp * 25 + vw];
    Db[t] = val;
  }
}

template <int P>
static constexpr size_t assemble3_smem() {
  return sizeof(double) * ((size_t)(P + 1) * (P + 1) * (P + 1) * (75 + 25) + 6 * (P + 1) * (P + 1) * 25);
}

void launch_assemble3(const Ctx& c, const LevelDev& L, const double* q, const double* d_dtau, double inv_odt,
                      cudaStream_t s) {
  const int* nbr = c.d_faces + 5 * c.n_faces;
#define PMG_A3(PP)                                                                                 \
  assemble3_kernel<PP><<<c.E, 128, assemble3_smem<PP>(), s>>>(c.E, q, L.met, L.face, nbr, L.op, c.ph, \
                                                               d_dtau, inv_odt, L.Dfull)
  switch (L.P) {
    case 0: PMG_A3(0); break;
    case 1: PMG_A3(1); break;
    case 2: PMG_A3(2); break;
    default: PMG_A3(3); break;
  }
#undef PMG_A3
  if (c.ph.mu > 0.0) launch_assemble_visc3(c, L, q, s);
}

template <class W, int P>
__global__ void __launch_bounds__(64) apply3_kernel(int E, const W* __restrict__ Dinv, const double* __restrict__ rs,
                                                    const double* __restrict__ cs, const double* __restrict__ r,
                                                    double* __restrict__ x, int accumulate) {
  constexpr int N = (P + 1) * (P + 1) * (P + 1), n = 5 * N;
  constexpr int EPB = N <= 32 ? 64 / N : 1;
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[EPB][n];
  const int le = threadIdx.x / N, pt = threadIdx.x - le * N;
  const int e = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (e < E);
  const size_t plane = (size_t)E * N;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v)
      sr[le][v * N + pt] = scaled_in<W>(r[v * plane + (size_t)e * N + pt], rs[(size_t)e * n + v * N + pt]);
  }
  __syncthreads();
  if (!active) return;
  Acc acc[5] = {0, 0, 0, 0, 0};
  const W* Dm = Dinv + (size_t)e * n * n + pt;
  for (int k = 0; k < n; ++k) {
    const Acc rk = sr[le][k];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = fma(blk_val(__ldg(Dm + (size_t)k * n + v * N)), rk, acc[v]);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double xv = scaled_out<W>(acc[v], cs[(size_t)e * n + v * N + pt]);
    const size_t o = v * plane + (size_t)e * N + pt;
    if (accumulate) x[o] += xv;
    else x[o] = xv;
  }
}

template <class W>
static void apply3_dispatch(const Ctx& c, const LevelDev& L, const double* r, double* x, int acc, cudaStream_t s) {
  const W* Dinv = (const W*)L.Dinv;
  const int N = L.N;
  const int epb = N <= 32 ? 64 / N : 1;
  const int threads = (epb * N + 31) / 32 * 32, blocks = (c.E + epb - 1) / epb;
#define PMG_AP3(PP) apply3_kernel<W, PP><<<blocks, threads, 0, s>>>(c.E, Dinv, L.rs, L.cs, r, x, acc)
  switch (L.P) {
    case 0: PMG_AP3(0); break;
    case 1: PMG_AP3(1); break;
    case 2: PMG_AP3(2); break;
    default: PMG_AP3(3); break;
  }
#undef PMG_AP3
}

void launch_apply3(const Ctx& c, const LevelDev& L, int prec, const double* r, double* x, int accumulate,
                   cudaStream_t s) {
  if (prec == PMG_PREC_FP64) apply3_dispatch<double>(c, L, r, x, accumulate, s);
  else if (prec == PMG_PREC_BF16R) apply3_dispatch<__nv_bfloat16>(c, L, r, x, accumulate, s);
  else apply3_dispatch<float>(c, L, r, x, accumulate, s);
}

// Dynamic shared memory of the assembly kernels above 48 KB (P = 3).
cudaError_t prepare_kernels3(const Ctx& c) {
  for (int l = 0; l < c.cfg.n_levels; ++l) {
    cudaError_t e = cudaSuccess;
    switch (c.lev[l].P) {
      case 0: e = cudaFuncSetAttribute(assemble3_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble3_smem<0>()); break;
      case 1: e = cudaFuncSetAttribute(assemble3_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble3_smem<1>()); break;
      case 2: e = cudaFuncSetAttribute(assemble3_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble3_smem<2>()); break;
      default: e = cudaFuncSetAttribute(assemble3_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)assemble3_smem<3>()); break;
    }
    if (e != cudaSuccess) return e;
  }
  if (c.ph.mu > 0.0) return prepare_assemble_visc3();
  return cudaSuccess;
}

}  // namespace pmg
