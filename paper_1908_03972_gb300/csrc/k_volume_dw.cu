// k_volume_dw.cu -- the residual-and-update of an element-Jacobi sweep
// (volume_kernel with APPLY, k_residual.cu) in double-word arithmetic.
//
// The sweep q += cs .* (D^-1 (rs .* F)) is the smoother, and on the coarse
// levels it only drives the FAS corrections of Section 3; the binary64
// residual of the finest level (a separate evaluation) defines the converged
// state.  Forming F on the FP32 pipes (dword.cuh, ~2^-46 relative rounding)
// instead of in binary64 takes the kernel's longest chain, ~130 FP64
// instructions per thread at one FP64 warp-instruction per ~64 cycles per SM
// sub-partition, off the FP64 pipe.
//
// Same steps and CTA shape as the binary64 kernel: contravariant fluxes of
// the element's points, the face jumps (common flux minus the extrapolated
// flux polynomial), the divergence with the DG correction, the level-system
// epilogue F = R - (q_c(q) - q_c(q_ref)) / (omega dt) + src - S (q_c(q)
// itself without q_ref), then the block update.  The states hold gauge
// pressure; with p_ref = 0 (absolute pressure, p ~ 1/(gamma Ma^2) in the
// momentum flux) the binary64 kernel is used.
#include "sweep_common.cuh"

namespace pmg {

template <int P, class W>
__global__ void __launch_bounds__(256, 1) volume_apply_dw_kernel(
    int E, double* q, const double* __restrict__ met, const double* __restrict__ Fcom, OpTabW opw, PhysW k,
    double inv_odt, const double* __restrict__ src, const double* __restrict__ S, const double* __restrict__ qref,
    const W* __restrict__ Dinv, const double* __restrict__ rs, const double* __restrict__ cs,
    double* __restrict__ werr) {
  constexpr int n1 = P + 1, N = n1 * n1, EPB = ElemsPerBlock<P>::value, n = 4 * N;
  using PF = VolPrefetch<P, W>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) unsigned long long mbar[2];   // 0: face fluxes, 1: blocks and scales
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[EPB][n];
  __shared__ dw sFt[EPB][4][N];
  __shared__ dw sGt[EPB][4][N];
  __shared__ dw sJ[EPB][4][4][n1];   // [face][var][k]
  __shared__ dw sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];

  const int le = threadIdx.x / N, pt = threadIdx.x - le * N;
  const int e = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (e < E);
  const size_t plane = (size_t)E * N;
  const size_t fplane = (size_t)E * 4 * n1;
  W* sDinv = reinterpret_cast<W*>(dsm);
  double* srs = reinterpret_cast<double*>(dsm + PF::dinv_bytes);
  double* scs = srs + EPB * n;
  double* sFc = scs + EPB * n;   // [v][local element][face][k]
  if (threadIdx.x == 0) {
    const int e0 = blockIdx.x * EPB, ne = min(EPB, E - e0);
    const unsigned bF = (unsigned)(ne * 4 * n1 * sizeof(double));
    const unsigned bS = (unsigned)(ne * n * sizeof(double));
    const unsigned bD = PF::blocks ? (unsigned)((size_t)ne * n * n * sizeof(W)) : 0u;
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    mbar_arrive_expect(&mbar[0], 4 * bF);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      bulk_g2s(sFc + v * EPB * 4 * n1, Fcom + v * fplane + (size_t)e0 * 4 * n1, bF, &mbar[0]);
    mbar_arrive_expect(&mbar[1], 2 * bS + bD);
    bulk_g2s(srs, rs + (size_t)e0 * n, bS, &mbar[1]);
    bulk_g2s(scs, cs + (size_t)e0 * n, bS, &mbar[1]);
    if (PF::blocks) bulk_g2s(sDinv, Dinv + (size_t)e0 * n * n, bD, &mbar[1]);
  }
  const size_t gi = (size_t)e * N + pt;
  // Sv: src - S of the epilogue
  double qq[4] = {0, 0, 0, 0}, qo[4] = {0, 0, 0, 0}, Sv[4] = {0, 0, 0, 0}, mt[5] = {0, 0, 0, 0, 0};
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qq[v] = q[v * plane + gi];
      if (qref) qo[v] = __ldg(qref + v * plane + gi);
      if (src) Sv[v] = __ldg(src + v * plane + gi);
      if (S) Sv[v] -= __ldg(S + v * plane + gi);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = __ldg(met + c * plane + gi);
  }
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = opw.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = opw.gL[threadIdx.x];
    sgR[threadIdx.x] = opw.gR[threadIdx.x];
    slm[threadIdx.x] = opw.lm[threadIdx.x];
    slp[threadIdx.x] = opw.lp[threadIdx.x];
  }

  dw Q[4], rho = {0.0f, 0.0f};
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) Q[v] = dw_from_double(qq[v]);   // gauge p, u, v, T
    rho = (Q[0] + k.p_ref) * rcp(Q[3]);
    const dw a = dw_from_double(mt[0]), b = dw_from_double(mt[1]);
    const dw c = dw_from_double(mt[2]), d = dw_from_double(mt[3]);
    const dw H = k.Cp * Q[3] + half(Q[1] * Q[1] + Q[2] * Q[2]);
    const dw mx = rho * Q[1], my = rho * Q[2];
    // Cartesian fluxes with the gauge pressure in the momentum rows
    const dw f[4] = {mx, mx * Q[1] + Q[0], mx * Q[2], mx * H};
    const dw g[4] = {my, my * Q[1], my * Q[2] + Q[0], my * H};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dw_acc x, y;
      x.add_prod(a, f[v]);
      x.add_prod(b, g[v]);
      y.add_prod(c, f[v]);
      y.add_prod(d, g[v]);
      sFt[le][v][pt] = x.value();
      sGt[le][v][pt] = y.value();
    }
  }
  __syncthreads();
  const bool okF = mbar_wait0(&mbar[0], k.wait_ns);
  if (!okF) *werr = 1.0;
  if (active) {
    for (int it = pt; it < 16 * n1; it += N) {
      const int f = it / (4 * n1), r = it - f * 4 * n1, v = r / n1, kk = r - v * n1;
      const bool xi = (f == 1 || f == 3);
      const bool plus = (f == 1 || f == 2);
      dw_acc loc;
#pragma unroll
      for (int m = 0; m < n1; ++m)
        loc.add_prod(plus ? slp[m] : slm[m], xi ? sFt[le][v][kk * n1 + m] : sGt[le][v][m * n1 + kk]);
      const double com = okF ? sFc[((v * EPB + le) * 4 + f) * n1 + kk]
                             : __ldg(Fcom + v * fplane + ((size_t)e * 4 + f) * n1 + kk);
      const dw cw = dw_from_double(plus ? com : -com);
      sJ[le][f][v][kk] = cw - loc.value();
    }
  }
  __syncthreads();
  const bool okS = mbar_wait0(&mbar[1], k.wait_ns);
  if (!okS) *werr = 1.0;
  if (active) {
    const int i = pt % n1, j = pt / n1;
    dw qc[4];
    if (qref) {
      // q_c(q) - q_c(q_ref), energy through p / (gamma - 1) + rho |v|^2 / 2
      // with the gauge-pressure difference (no p ~ 1/Ma^2 is rounded)
      dw Qo[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) Qo[v] = dw_from_double(qo[v]);
      const dw rhoo = (Qo[0] + k.p_ref) * rcp(Qo[3]);
      qc[0] = rho - rhoo;
      qc[1] = rho * Q[1] - rhoo * Qo[1];
      qc[2] = rho * Q[2] - rhoo * Qo[2];
      qc[3] = (Q[0] - Qo[0]) * k.inv_gm1 +
              half(rho * (Q[1] * Q[1] + Q[2] * Q[2]) - rhoo * (Qo[1] * Qo[1] + Qo[2] * Qo[2]));
    } else {
      qc[0] = rho;
      qc[1] = rho * Q[1];
      qc[2] = rho * Q[2];
      qc[3] = rho * (Q[3] * k.inv_gm1 + half(Q[1] * Q[1] + Q[2] * Q[2]));
    }
    const dw invJ = dw_from_double(mt[4]);
    const dw nodt = dw_from_double(-inv_odt);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dw_acc acc;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        acc.add_prod(sD[i][m], sFt[le][v][j * n1 + m]);
        acc.add_prod(sD[j][m], sGt[le][v][m * n1 + i]);
      }
      acc.add_prod(sgL[i], sJ[le][3][v][j]);
      acc.add_prod(sgR[i], sJ[le][1][v][j]);
      acc.add_prod(sgL[j], sJ[le][0][v][i]);
      acc.add_prod(sgR[j], sJ[le][2][v][i]);
      // F = -acc / |J| - qc / (omega dt) + src - S
      dw_acc F;
      F.add_prod(-acc.value(), invJ);
      F.add_prod(qc[v], nodt);
      F.add(dw_from_double(Sv[v]));
      const int row = v * N + pt;
      sr[le][row] = scaled_in_dw<W>(F.value(), okS ? srs[le * n + row] : rs[(size_t)e * n + row]);
    }
  }
  __syncthreads();
  if (active) {
    // thread (le, pt) owns rows 4 pt .. 4 pt + 3 of its element's block
    Acc acc[4] = {0, 0, 0, 0};
    if (PF::blocks && okS) {
      const W* Dm = sDinv + (size_t)le * n * n + 4 * pt;
#pragma unroll 8
      for (int kk = 0; kk < n; ++kk) {
        const Acc rk = sr[le][kk];
        Acc d[4];
        ld4(Dm + (size_t)kk * n, d);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = fma(d[m], rk, acc[m]);
      }
    } else {
      const W* Dm = Dinv + (size_t)e * n * n + 4 * pt;
#pragma unroll 8
      for (int kk = 0; kk < n; ++kk) {
        const Acc rk = sr[le][kk];
        Acc d[4];
        ldg4(Dm + (size_t)kk * n, d);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = fma(d[m], rk, acc[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int row = 4 * pt + m;
      const int v = row / N, p2 = row - v * N;
      const size_t o = v * plane + (size_t)e * N + p2;
      const double csc = okS ? scs[le * n + row] : cs[(size_t)e * n + row];
      q[o] = q[o] + scaled_out<W>(acc[m], csc);
    }
  }
  // copies still in flight land before the CTA exits
  if (!okF) mbar_drain0(&mbar[0]);
  if (!okS) mbar_drain0(&mbar[1]);
}

template <class W>
static void dw_dispatch(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                        const double* S, const double* qref, cudaStream_t s) {
  const int threads = residual_threads_per_block(L.P), blocks = residual_blocks_for(L.P, c.E);
  const W* Dinv = (const W*)L.Dinv;
#define PMG_VDW(PP)                                                                                         \
  volume_apply_dw_kernel<PP, W><<<blocks, threads, VolPrefetch<PP, W>::smem, s>>>(                          \
      c.E, q, L.met, L.Fcom, L.opw, c.phw, inv_odt, src, S, qref, Dinv, L.rs, L.cs, c.d_scal + 1)
  switch (L.P) {
    case 0: PMG_VDW(0); break;
    case 1: PMG_VDW(1); break;
    case 2: PMG_VDW(2); break;
    case 3: PMG_VDW(3); break;
    case 4: PMG_VDW(4); break;
    default: PMG_VDW(5); break;
  }
#undef PMG_VDW
}

bool volume_dw_applies(const Ctx& c) {
  return c.dim == 2 && flux_dw_sweep(c) && c.ph.mu == 0.0 && c.ph.p_ref != 0.0;
}

void launch_volume_apply_dw(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                            const double* S, const double* qref, int prec, cudaStream_t s) {
  if (prec == PMG_PREC_FP64) dw_dispatch<double>(c, L, q, inv_odt, src, S, qref, s);
  else if (prec == PMG_PREC_BF16R) dw_dispatch<__nv_bfloat16>(c, L, q, inv_odt, src, S, qref, s);
  else dw_dispatch<float>(c, L, q, inv_odt, src, S, qref, s);
}

template <class W>
static cudaError_t prep_dw(int P) {
#define PMG_PDW(PP)                                                                                       \
  return cudaFuncSetAttribute(volume_apply_dw_kernel<PP, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                              (int)VolPrefetch<PP, W>::smem)
  switch (P) {
    case 0: PMG_PDW(0);
    case 1: PMG_PDW(1);
    case 2: PMG_PDW(2);
    case 3: PMG_PDW(3);
    case 4: PMG_PDW(4);
    default: PMG_PDW(5);
  }
#undef PMG_PDW
}

cudaError_t prepare_volume_dw_kernels(const Ctx& c) {
  for (int l = 0; l < c.cfg.n_levels; ++l) {
    cudaError_t e = c.cfg.block_prec == PMG_PREC_FP64    ? prep_dw<double>(c.lev[l].P)
                    : c.cfg.block_prec == PMG_PREC_BF16R ? prep_dw<__nv_bfloat16>(c.lev[l].P)
                                                         : prep_dw<float>(c.lev[l].P);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pmg
