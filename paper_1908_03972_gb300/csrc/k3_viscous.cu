// k3_viscous.cu -- viscous part of the element blocks on hexahedra (Section
// 2.1 viscous fluxes; Section 2.3 eq. com_q and the BR2 common gradient of
// eq. com_grad_q, d = 3).
//
// assemble_visc3 adds the viscous part of -dR_e/dq_e to the blocks the
// inviscid assembly (k3_blocks.cu) wrote, one CTA per element.  Only
// (u, v, w, T) enter the viscous fluxes, so 4 N of the 5 N columns and rows
// 1..4 are touched.  The columns are exact tangents -- dual numbers through
// the residual's viscous flux (physics3.cuh viscous_flux3) -- of the
// element's viscous residual with neighbour data frozen:
//  (A) at every solution point, the tangent of the corrected gradient
//      (Lagrange derivative plus the DG correction of d(q_com - q^-) =
//      kappa dq^- on the two faces of each line; kappa = -1/2 on interior
//      and far-field faces, -1 for the velocity and 0 for the temperature at
//      no-slip walls) and of the velocity, hence of the viscous flux, turned
//      into the contravariant fluxes with J a^i;
//  (B) at every face point, the tangent of the common viscous flux (q_com
//      and the BR2 common gradient: half the own broken-gradient tangent, or
//      all of it where a boundary mirrors the element, plus the lifting of
//      d(q^+ - q^-) = 2 kappa dq^-) minus the extrapolated flux tangent;
//  (C) derivative plus DG correction along the three lines, times -1/|J|.
// Columns are processed C at a time; everything lives in dynamic shared
// memory.
#include "pmg_internal.h"
#include "physics3.cuh"

namespace pmg {

template <int P>
struct Visc3 {
  static constexpr int n1 = P + 1, N = n1 * n1 * n1, NF = n1 * n1, FP = 6 * NF;
  static constexpr int kThreads = 256;
  static constexpr int C0 = kThreads / (N > FP ? N : FP);
  static constexpr int C = C0 < 1 ? 1 : (C0 > 4 * N ? 4 * N : C0);   // columns per pass
  // fixed arrays: sV 4N, sM 10N, sGb 12N, sGc 12N, sDq 4FP, sQc 3FP, sGf 12FP, sS 5FP
  static constexpr size_t fixed = (size_t)38 * N + (size_t)24 * FP;
  // per column: sdF 3*4*N, sdJ 6*4*NF
  static constexpr size_t per_col = (size_t)12 * N + (size_t)24 * NF;
  static constexpr size_t smem = sizeof(double) * (fixed + C * per_col);
};

template <int P>
__device__ __forceinline__ int lpt3(int f, int a, int b, int m) {
  constexpr int n1 = P + 1;
  const int d = f >> 1;
  const int i = d == 0 ? m : a, j = d == 1 ? m : (d == 0 ? a : b), k = d == 2 ? m : b;
  return (k * n1 + j) * n1 + i;
}

template <int P>
__global__ void __launch_bounds__(256) assemble_visc3_kernel(int E, const double* __restrict__ q,
                                                             const double* __restrict__ Gb,
                                                             const double* __restrict__ met,
                                                             const double* __restrict__ face,
                                                             const double* __restrict__ fJinv,
                                                             const int* __restrict__ nbr, OpTab op, Phys ph,
                                                             double* __restrict__ Dout) {
  using T3 = Visc3<P>;
  constexpr int n1 = T3::n1, N = T3::N, NF = T3::NF, FP = T3::FP, n = 5 * N, C = T3::C;
  extern __shared__ __align__(16) double dyn[];
  double* sV = dyn;                 // [4][N]   u, v, w, T
  double* sM = sV + 4 * N;          // [10][N]  J a^i_c (3 i + c), 1/|J|
  double* sGb = sM + 10 * N;        // [12][N]  broken gradient (c*4 + k)
  double* sGc = sGb + 12 * N;       // [12][N]  corrected gradient
  double* sDq = sGc + 12 * N;       // [FP][4]  q^+ - q^- of (u, v, w, T)
  double* sQc = sDq + 4 * FP;       // [FP][3]  q_com velocity
  double* sGf = sQc + 3 * FP;       // [FP][12] common gradient (first: the neighbour's trace)
  double* sS = sGf + 12 * FP;       // [FP][5]  unit normal, area, lifting weight
  double* sdF = sS + 5 * FP;        // [C][3][4][N] tangents of the viscous contravariant fluxes
  double* sdJ = sdF + C * 12 * N;   // [C][6][4][NF] tangents of the face jumps
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  __shared__ double sKap[6][4];
  __shared__ int sBc[6];
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t plane = (size_t)E * N;
  for (int t = tid; t < N; t += nt) {
#pragma unroll
    for (int k = 0; k < 4; ++k) sV[k * N + t] = q[(k + 1) * plane + (size_t)e * N + t];
#pragma unroll
    for (int c = 0; c < 10; ++c) sM[c * N + t] = met[c * plane + (size_t)e * N + t];
  }
  if (tid < n1 * n1) sD[tid / n1][tid % n1] = op.D[tid / n1][tid % n1];
  if (tid < n1) {
    sgL[tid] = op.gL[tid];
    sgR[tid] = op.gR[tid];
    slm[tid] = op.lm[tid];
    slp[tid] = op.lp[tid];
  }
  if (tid < 6) {
    const int en = nbr[(e * 6 + tid) * 3], bc = nbr[(e * 6 + tid) * 3 + 1];
    sBc[tid] = en < 0 ? bc : 0;
    const bool wall = en < 0 && bc == PMG_BC_NOSLIP_WALL;
    sKap[tid][0] = sKap[tid][1] = sKap[tid][2] = wall ? -1.0 : -0.5;
    sKap[tid][3] = wall ? 0.0 : -0.5;
  }
  __syncthreads();
  // values: own broken gradients
  for (int t = tid; t < N; t += nt) {
    const int i = t % n1, j = (t / n1) % n1, k = t / (n1 * n1);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const double* V = sV + w * N;
      const double r0 = V[(k * n1 + j) * n1], r1 = V[k * n1 * n1 + i], r2 = V[j * n1 + i];
      double dr[3] = {0.0, 0.0, 0.0};
      for (int m = 0; m < n1; ++m) {
        dr[0] = fma(sD[i][m], V[(k * n1 + j) * n1 + m] - r0, dr[0]);
        dr[1] = fma(sD[j][m], V[(k * n1 + m) * n1 + i] - r1, dr[1]);
        dr[2] = fma(sD[k][m], V[(m * n1 + j) * n1 + i] - r2, dr[2]);
      }
      for (int c = 0; c < 3; ++c)
        sGb[(c * 4 + w) * N + t] =
            sM[9 * N + t] * (sM[(0 + c) * N + t] * dr[0] + sM[(3 + c) * N + t] * dr[1] + sM[(6 + c) * N + t] * dr[2]);
    }
  }
  // values: traces, jumps and frozen neighbour data at the face points
  for (int t = tid; t < FP; t += nt) {
    const int f = t / NF, fp = t - f * NF, a = fp % n1, b = fp / n1;
    const bool plus = f & 1;
    const int en = nbr[(e * 6 + f) * 3], fn = nbr[(e * 6 + f) * 3 + 1], o = nbr[(e * 6 + f) * 3 + 2];
    const bool bnd = en < 0;
    int a2 = 0, b2 = 0;
    if (!bnd) {
      const int s = (o & 4) ? b : a, tt = (o & 4) ? a : b;
      a2 = (o & 1) ? P - s : s;
      b2 = (o & 2) ? P - tt : tt;
    }
    double qm[4], qp[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const double ref = sV[w * N];
      double sm = 0.0, sp = 0.0;
      for (int m = 0; m < n1; ++m) {
        sm = fma(plus ? slp[m] : slm[m], sV[w * N + lpt3<P>(f, a, b, m)] - ref, sm);
        if (!bnd)
          sp = fma((fn & 1) ? slp[m] : slm[m], q[(w + 1) * plane + (size_t)en * N + lpt3<P>(fn, a2, b2, m)] - ref,
                   sp);
      }
      qm[w] = ref + sm;
      qp[w] = ref + sp;
    }
    if (bnd) {   // far field: the free stream; no-slip wall: velocity reversed, same T
      for (int w = 0; w < 4; ++w) qp[w] = fn == PMG_BC_FARFIELD ? ph.qinf[w + 1] : (w < 3 ? -qm[w] : qm[w]);
    }
    for (int w = 0; w < 4; ++w) sDq[t * 4 + w] = qp[w] - qm[w];
    for (int c = 0; c < 3; ++c) sQc[t * 3 + c] = 0.5 * (qm[c] + qp[c]);
    for (int c = 0; c < 12; ++c) {
      double s = 0.0;
      if (!bnd)
        for (int m = 0; m < n1; ++m)
          s = fma((fn & 1) ? slp[m] : slm[m], Gb[c * plane + (size_t)en * N + lpt3<P>(fn, a2, b2, m)], s);
      sGf[t * 12 + c] = s;
    }
    const double* g = face + (((size_t)e * 6 + f) * NF + fp) * 4;
    const double iJm = fJinv[((size_t)e * 6 + f) * NF + fp];
    const double iJp = bnd ? iJm : fJinv[((size_t)en * 6 + fn) * NF + b2 * n1 + a2];
    sS[t * 5 + 0] = g[0];
    sS[t * 5 + 1] = g[1];
    sS[t * 5 + 2] = g[2];
    sS[t * 5 + 3] = g[3];
    sS[t * 5 + 4] = 0.25 * op.pen * (iJm + iJp) * g[3];
  }
  __syncthreads();
  // values: corrected gradients at the solution points, common gradients
  for (int t = tid; t < N; t += nt) {
    const int i = t % n1, j = (t / n1) % n1, k = t / (n1 * n1);
    const int idx[3] = {i, j, k}, fpd[3] = {k * n1 + j, k * n1 + i, j * n1 + i};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const double* V = sV + w * N;
      const double r0 = V[(k * n1 + j) * n1], r1 = V[k * n1 * n1 + i], r2 = V[j * n1 + i];
      double dr[3] = {0.0, 0.0, 0.0};
      for (int m = 0; m < n1; ++m) {
        dr[0] = fma(sD[i][m], V[(k * n1 + j) * n1 + m] - r0, dr[0]);
        dr[1] = fma(sD[j][m], V[(k * n1 + m) * n1 + i] - r1, dr[1]);
        dr[2] = fma(sD[k][m], V[(m * n1 + j) * n1 + i] - r2, dr[2]);
      }
      for (int d = 0; d < 3; ++d) {
        dr[d] = fma(sgL[idx[d]], 0.5 * sDq[((2 * d) * NF + fpd[d]) * 4 + w], dr[d]);
        dr[d] = fma(sgR[idx[d]], 0.5 * sDq[((2 * d + 1) * NF + fpd[d]) * 4 + w], dr[d]);
      }
      for (int c = 0; c < 3; ++c)
        sGc[(c * 4 + w) * N + t] =
            sM[9 * N + t] * (sM[(0 + c) * N + t] * dr[0] + sM[(3 + c) * N + t] * dr[1] + sM[(6 + c) * N + t] * dr[2]);
    }
  }
  for (int t = tid; t < FP; t += nt) {
    const int f = t / NF, fp = t - f * NF, a = fp % n1, b = fp / n1;
    const bool plus = f & 1;
    for (int c = 0; c < 12; ++c) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) s = fma(plus ? slp[m] : slm[m], sGb[c * N + lpt3<P>(f, a, b, m)], s);
      const double other = sBc[f] ? s : sGf[t * 12 + c];   // a boundary mirrors the element
      sGf[t * 12 + c] = fma(sS[t * 5 + 4] * sS[t * 5 + c / 4], sDq[t * 4 + c % 4], 0.5 * (s + other));
    }
  }
  __syncthreads();

  double* Db = Dout + (size_t)e * n * n;
  for (int c0 = 0; c0 < 4 * N; c0 += C) {
    // (A) tangents of the viscous contravariant fluxes at the solution points
    for (int t = tid; t < C * N; t += nt) {
      const int cc = t / N, pt = t - cc * N, col = c0 + cc;
      if (col >= 4 * N) continue;
      const int w = col / N, cp = col - w * N;
      const int ci = cp % n1, cj = (cp / n1) % n1, ck = cp / (n1 * n1);
      const int i = pt % n1, j = (pt / n1) % n1, k = pt / (n1 * n1);
      // d(corrected reference derivative along direction d)/dq_w(cp)
      double ddr[3];
      ddr[0] = (cj == j && ck == k) ? sD[i][ci] + sgL[i] * sKap[0][w] * slm[ci] + sgR[i] * sKap[1][w] * slp[ci] : 0.0;
      ddr[1] = (ci == i && ck == k) ? sD[j][cj] + sgL[j] * sKap[2][w] * slm[cj] + sgR[j] * sKap[3][w] * slp[cj] : 0.0;
      ddr[2] = (ci == i && cj == j) ? sD[k][ck] + sgL[k] * sKap[4][w] * slm[ck] + sgR[k] * sKap[5][w] * slp[ck] : 0.0;
      const double iJ = sM[9 * N + pt];
      Dual gr[12];
      for (int c = 0; c < 3; ++c) {
        const double dg =
            iJ * (sM[(0 + c) * N + pt] * ddr[0] + sM[(3 + c) * N + pt] * ddr[1] + sM[(6 + c) * N + pt] * ddr[2]);
        for (int kk = 0; kk < 4; ++kk) gr[c * 4 + kk] = Dual(sGc[(c * 4 + kk) * N + pt], kk == w ? dg : 0.0);
      }
      Dual uvw[3];
      for (int c = 0; c < 3; ++c) uvw[c] = Dual(sV[c * N + pt], (w == c && cp == pt) ? 1.0 : 0.0);
      Dual fv[12];
      viscous_flux3(uvw, gr, ph, fv);
      for (int d = 0; d < 3; ++d)
        for (int r = 0; r < 4; ++r)
          sdF[((cc * 3 + d) * 4 + r) * N + pt] =
              -(sM[(3 * d + 0) * N + pt] * fv[r].d + sM[(3 * d + 1) * N + pt] * fv[4 + r].d +
                sM[(3 * d + 2) * N + pt] * fv[8 + r].d);
    }
    __syncthreads();
    // (B) tangents of the face jumps: common minus extrapolated flux
    for (int t = tid; t < C * FP; t += nt) {
      const int cc = t / FP, tf = t - cc * FP, col = c0 + cc;
      if (col >= 4 * N) continue;
      const int w = col / N, cp = col - w * N;
      const int cidx[3] = {cp % n1, (cp / n1) % n1, cp / (n1 * n1)};
      const int f = tf / NF, fp = tf - f * NF, a = fp % n1, b = fp / n1, d = f >> 1;
      const bool plus = f & 1;
      const double* l = plus ? slp : slm;
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;   // tangential directions: (a, b)
      const bool on_line = cidx[t1] == a && cidx[t2] == b;
      const double dqm = on_line ? l[cidx[d]] : 0.0;
      // trace of the broken-gradient tangent along the normal line
      double dg[3] = {0.0, 0.0, 0.0};
      for (int m = 0; m < n1; ++m) {
        const int p2 = lpt3<P>(f, a, b, m);
        const int pidx[3] = {p2 % n1, (p2 / n1) % n1, p2 / (n1 * n1)};
        double bd[3];
        bd[0] = (cidx[1] == pidx[1] && cidx[2] == pidx[2]) ? sD[pidx[0]][cidx[0]] : 0.0;
        bd[1] = (cidx[0] == pidx[0] && cidx[2] == pidx[2]) ? sD[pidx[1]][cidx[1]] : 0.0;
        bd[2] = (cidx[0] == pidx[0] && cidx[1] == pidx[1]) ? sD[pidx[2]][cidx[2]] : 0.0;
        const double iJ = sM[9 * N + p2];
        for (int c = 0; c < 3; ++c)
          dg[c] = fma(l[m], iJ * (sM[(0 + c) * N + p2] * bd[0] + sM[(3 + c) * N + p2] * bd[1] +
                                  sM[(6 + c) * N + p2] * bd[2]), dg[c]);
      }
      const double* S = sS + tf * 5;
      const double kap = sKap[f][w], gfac = sBc[f] ? 1.0 : 0.5;
      Dual gr[12];
      for (int c = 0; c < 3; ++c)
        for (int kk = 0; kk < 4; ++kk)
          gr[c * 4 + kk] =
              Dual(sGf[tf * 12 + c * 4 + kk], kk == w ? fma(2.0 * kap * S[4] * S[c], dqm, gfac * dg[c]) : 0.0);
      Dual uvw[3];
      for (int c = 0; c < 3; ++c) uvw[c] = Dual(sQc[tf * 3 + c], w == c ? (1.0 + kap) * dqm : 0.0);
      Dual fv[12];
      viscous_flux3(uvw, gr, ph, fv);
      const int nr = (sBc[f] && sBc[f] != PMG_BC_FARFIELD) ? 3 : 4;   // walls: no viscous energy flux
      for (int r = 0; r < 4; ++r) {
        const double dcom = r < nr ? -(fv[r].d * S[0] + fv[4 + r].d * S[1] + fv[8 + r].d * S[2]) * S[3] : 0.0;
        double loc = 0.0;
        for (int m = 0; m < n1; ++m) loc = fma(l[m], sdF[((cc * 3 + d) * 4 + r) * N + lpt3<P>(f, a, b, m)], loc);
        sdJ[((cc * 6 + f) * 4 + r) * NF + fp] = (plus ? dcom : -dcom) - loc;
      }
    }
    __syncthreads();
    // (C) tangent of the residual: derivative plus correction, scaled by -1/|J|
    for (int t = tid; t < C * N; t += nt) {
      const int cc = t / N, pt = t - cc * N, col = c0 + cc;
      if (col >= 4 * N) continue;
      const int w = col / N, cp = col - w * N;
      const int i = pt % n1, j = (pt / n1) % n1, k = pt / (n1 * n1);
      for (int r = 0; r < 4; ++r) {
        const double* F0 = sdF + ((cc * 3 + 0) * 4 + r) * N;
        const double* F1 = sdF + ((cc * 3 + 1) * 4 + r) * N;
        const double* F2 = sdF + ((cc * 3 + 2) * 4 + r) * N;
        const double* Jf = sdJ + (size_t)(cc * 6) * 4 * NF + r * NF;   // face f at Jf + f * 4 * NF
        double acc = 0.0;
        for (int m = 0; m < n1; ++m) {
          acc = fma(sD[i][m], F0[(k * n1 + j) * n1 + m], acc);
          acc = fma(sD[j][m], F1[(k * n1 + m) * n1 + i], acc);
          acc = fma(sD[k][m], F2[(m * n1 + j) * n1 + i], acc);
        }
        acc = fma(sgL[i], Jf[0 * 4 * NF + k * n1 + j], acc);
        acc = fma(sgR[i], Jf[1 * 4 * NF + k * n1 + j], acc);
        acc = fma(sgL[j], Jf[2 * 4 * NF + k * n1 + i], acc);
        acc = fma(sgR[j], Jf[3 * 4 * NF + k * n1 + i], acc);
        acc = fma(sgL[k], Jf[4 * 4 * NF + j * n1 + i], acc);
        acc = fma(sgR[k], Jf[5 * 4 * NF + j * n1 + i], acc);
        const double dR = -acc * sM[9 * N + pt];
        Db[(size_t)((r + 1) * N + pt) * n + (w + 1) * N + cp] -= dR;   // D = ... - dR/dq
      }
    }
    __syncthreads();
  }
}

template <int P>
static cudaError_t prepare_visc3() {
  return cudaFuncSetAttribute(assemble_visc3_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Visc3<P>::smem);
}

cudaError_t prepare_assemble_visc3() {
  cudaError_t e = prepare_visc3<0>();
  if (e == cudaSuccess) e = prepare_visc3<1>();
  if (e == cudaSuccess) e = prepare_visc3<2>();
  if (e == cudaSuccess) e = prepare_visc3<3>();
  return e;
}

void launch_assemble_visc3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s) {
  launch_grad3(c, L, q, s);
  const int* nbr = c.d_faces + 5 * c.n_faces;
#define PMG_AV3(PP)                                                                                          \
  assemble_visc3_kernel<PP><<<c.E, Visc3<PP>::kThreads, Visc3<PP>::smem, s>>>(c.E, q, L.Gb, L.met, L.face, \
                                                                              L.fJinv, nbr, L.op, c.ph, L.Dfull)
  switch (L.P) {
    case 0: PMG_AV3(0); break;
    case 1: PMG_AV3(1); break;
    case 2: PMG_AV3(2); break;
    default: PMG_AV3(3); break;
  }
#undef PMG_AV3
}

}  // namespace pmg
