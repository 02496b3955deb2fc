// k_viscous.cu -- viscous terms of the FR residual and of the element blocks
// (Section 2.1 viscous fluxes; Section 2.3 common solution, eq. com_q, and
// BR2 common gradient, eq. com_grad_q).
//
//  * grad: broken (uncorrected) gradients of (u, v, T) at every solution
//    point, by the Lagrange derivative and the chain rule with the metric
//    terms.  The face launch extrapolates them to both sides of each face.
//  * assemble_visc: adds the viscous part of -dR_e/dq_e to the element
//    blocks that the inviscid assembly wrote.  Only u, v and T enter the
//    viscous fluxes, so 3 N of the 4 N columns are touched.  The columns are
//    exact tangents (dual numbers through the same viscous flux code as the
//    residual) of the element's viscous residual with neighbour data frozen:
//    corrected gradients at the solution points, BR2 common gradient and
//    q_com at the flux points, divergence and DG correction.  On boundary
//    faces the ghost state follows the own trace: q_com - q^- changes by
//    kappa dq^- (kappa = -1/2 for interior and far-field faces, -1 for the
//    velocity and 0 for the temperature at no-slip adiabatic walls), and the
//    mirrored gradient trace doubles the own gradient's share.
#include "pmg_internal.h"

namespace pmg {

// ----------------------------------------------------------------- gradients
// Broken gradient of (u, v, T): Gb[c * 3 + v] planes, c = x, y.  Derivatives
// are taken of the differences to the line's first value (the derivative
// matrix annihilates constants), which keeps T ~ 1/Ma^2 out of the rounding.
template <int P>
__global__ void __launch_bounds__(128) grad_kernel(int E, const double* __restrict__ q,
                                                   const double* __restrict__ met, OpTab op,
                                                   double* __restrict__ Gb) {
  constexpr int n1 = P + 1, N = n1 * n1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * N) return;
  const int e = tid / N, pt = tid - e * N, i = pt % n1, j = pt / n1;
  const size_t plane = (size_t)E * N;
  const double a = __ldg(met + tid), b = __ldg(met + plane + tid);
  const double c = __ldg(met + 2 * plane + tid), d = __ldg(met + 3 * plane + tid);
  const double iJ = __ldg(met + 4 * plane + tid);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const double* qv = q + (v + 1) * plane + (size_t)e * N;
    const double rx = __ldg(qv + j * n1), re = __ldg(qv + i);
    double ax = 0.0, ae = 0.0;
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      ax = fma(op.D[i][m], __ldg(qv + j * n1 + m) - rx, ax);
      ae = fma(op.D[j][m], __ldg(qv + m * n1 + i) - re, ae);
    }
    Gb[v * plane + tid] = iJ * fma(a, ax, c * ae);
    Gb[(3 + v) * plane + tid] = iJ * fma(b, ax, d * ae);
  }
}

void launch_grad(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s) {
  const int total = c.E * L.N, threads = 128, blocks = (total + threads - 1) / threads;
#define PMG_GRAD(PP) grad_kernel<PP><<<blocks, threads, 0, s>>>(c.E, q, L.met, L.op, L.Gb)
  switch (L.P) {
    case 0: PMG_GRAD(0); break;
    case 1: PMG_GRAD(1); break;
    case 2: PMG_GRAD(2); break;
    case 3: PMG_GRAD(3); break;
    case 4: PMG_GRAD(4); break;
    default: PMG_GRAD(5); break;
  }
#undef PMG_GRAD
}

// ------------------------------------------------------- viscous block part
// Columns processed together: one thread per (column, solution point) and
// per (column, face point).
template <int P>
struct ViscCols {
  static constexpr int N = (P + 1) * (P + 1), FP = 4 * (P + 1);
  static constexpr int value = 256 / (N > FP ? N : FP);
};

template <int P>
__global__ void __launch_bounds__(256) assemble_visc_kernel(int E, const double* __restrict__ q,
                                                            const double* __restrict__ Gb,
                                                            const double* __restrict__ met,
                                                            const double* __restrict__ face,
                                                            const double* __restrict__ fJinv,
                                                            const int* __restrict__ nbr, OpTab op, Phys ph,
                                                            double* __restrict__ Dout) {
  constexpr int n1 = P + 1, N = n1 * n1, n = 4 * N, FP = 4 * n1, C = ViscCols<P>::value;
  __shared__ double sV[3][N];       // u, v, T
  __shared__ double sM[5][N];       // metric terms a, b, c, d, 1/|J|
  __shared__ double sGb[6][N];      // broken gradient (values)
  __shared__ double sGc[6][N];      // corrected gradient (values)
  __shared__ double sDq[FP][3];     // q^+ - q^- of (u, v, T) at each face point
  __shared__ double sQc[FP][2];     // q_com velocities
  __shared__ double sGf[FP][6];     // common gradient (values)
  __shared__ double sS[FP][4];      // nx, ny, dS, lifting weight
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  __shared__ double sKap[4][3];     // d(q_com - q^-)/dq^- per face and variable (u, v, T)
  __shared__ int sBc[4];            // boundary type per face, 0 for interior faces
  __shared__ double sdF[C][3][N], sdG[C][3][N];   // tangents of the total contravariant fluxes, rows 1..3
  __shared__ double sdJ[C][4][3][n1];             // tangents of the face jumps
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t plane = (size_t)E * N;
  for (int t = tid; t < N; t += nt) {
#pragma unroll
    for (int v = 0; v < 3; ++v) sV[v][t] = q[(v + 1) * plane + (size_t)e * N + t];
#pragma unroll
    for (int k = 0; k < 5; ++k) sM[k][t] = met[k * plane + (size_t)e * N + t];
  }
  if (tid < n1 * n1) {
    const int i = tid / n1, m = tid % n1;
    sD[i][m] = op.D[i][m];
  }
  if (tid < 4) {
    const int en = nbr[(e * 4 + tid) * 3 + 0], bc = nbr[(e * 4 + tid) * 3 + 1];
    sBc[tid] = en < 0 ? bc : 0;
    const bool wall = en < 0 && bc == PMG_BC_NOSLIP_WALL;
    sKap[tid][0] = sKap[tid][1] = wall ? -1.0 : -0.5;
    sKap[tid][2] = wall ? 0.0 : -0.5;
  }
  if (tid < n1) {
    sgL[tid] = op.gL[tid];
    sgR[tid] = op.gR[tid];
    slm[tid] = op.lm[tid];
    slp[tid] = op.lp[tid];
  }
  __syncthreads();
  // values: own broken gradients; traces, jumps and frozen neighbour data
  for (int t = tid; t < N; t += nt) {
    const int i = t % n1, j = t / n1;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double ax = 0.0, ae = 0.0;
      for (int m = 0; m < n1; ++m) {
        ax = fma(sD[i][m], sV[v][j * n1 + m] - sV[v][j * n1], ax);
        ae = fma(sD[j][m], sV[v][m * n1 + i] - sV[v][i], ae);
      }
      sGb[v][t] = sM[4][t] * fma(sM[0][t], ax, sM[2][t] * ae);
      sGb[3 + v][t] = sM[4][t] * fma(sM[1][t], ax, sM[3][t] * ae);
    }
  }
  for (int t = tid; t < FP; t += nt) {
    const int f = t / n1, k = t - f * n1;
    const bool plus = (f == 1 || f == 2), eta = (f == 0 || f == 2);
    const int en = nbr[(e * 4 + f) * 3 + 0], fn = nbr[(e * 4 + f) * 3 + 1], rev = nbr[(e * 4 + f) * 3 + 2];
    const bool bnd = en < 0;
    const int kn = rev ? P - k : k;
    const bool pn = (fn == 1 || fn == 2), etan = (fn == 0 || fn == 2);
    const int stride = etan ? n1 : 1;
    const size_t nbase = bnd ? 0 : (size_t)en * N + (etan ? kn : kn * n1);
    const double* g = face + (((size_t)e * 4 + f) * n1 + k) * 3;
    double qm[3], qp[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double sm = 0.0, sp = 0.0;
      const double ref = sV[v][0];
      for (int m = 0; m < n1; ++m) {
        sm = fma(plus ? slp[m] : slm[m], sV[v][eta ? m * n1 + k : k * n1 + m] - ref, sm);
        if (!bnd) sp = fma(pn ? slp[m] : slm[m], q[(v + 1) * plane + nbase + m * stride] - ref, sp);
      }
      qm[v] = ref + sm;
      qp[v] = ref + sp;
      sDq[t][v] = sp - sm;
    }
    if (bnd) {   // ghost of (u, v, T); walls keep T, the far field is the free stream
      if (fn == PMG_BC_FARFIELD) {
        qp[0] = ph.qinf[1];
        qp[1] = ph.qinf[2];
        qp[2] = ph.qinf[3];
      } else {
        qp[0] = -qm[0];
        qp[1] = -qm[1];
        qp[2] = qm[2];
      }
      for (int v = 0; v < 3; ++v) sDq[t][v] = qp[v] - qm[v];
    }
    sQc[t][0] = 0.5 * (qm[0] + qp[0]);
    sQc[t][1] = 0.5 * (qm[1] + qp[1]);
#pragma unroll
    for (int c = 0; c < 6; ++c) {   // neighbour's broken-gradient trace, for now
      double s = 0.0;
      if (!bnd)
        for (int m = 0; m < n1; ++m) s = fma(pn ? slp[m] : slm[m], Gb[c * plane + nbase + m * stride], s);
      sGf[t][c] = s;
    }
    sS[t][0] = g[0];
    sS[t][1] = g[1];
    sS[t][2] = g[2];
    const double iJm = fJinv[((size_t)e * 4 + f) * n1 + k];
    const double iJp = bnd ? iJm : fJinv[((size_t)en * 4 + fn) * n1 + kn];
    sS[t][3] = 0.25 * op.pen * (iJm + iJp) * g[2];
  }
  __syncthreads();
  // values: corrected gradients at the solution points, common gradients
  for (int t = tid; t < N; t += nt) {
    const int i = t % n1, j = t / n1;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double ax = 0.0, ae = 0.0;
      for (int m = 0; m < n1; ++m) {
        ax = fma(sD[i][m], sV[v][j * n1 + m] - sV[v][j * n1], ax);
        ae = fma(sD[j][m], sV[v][m * n1 + i] - sV[v][i], ae);
      }
      ax = fma(sgL[i], 0.5 * sDq[3 * n1 + j][v], ax);
      ax = fma(sgR[i], 0.5 * sDq[1 * n1 + j][v], ax);
      ae = fma(sgL[j], 0.5 * sDq[0 * n1 + i][v], ae);
      ae = fma(sgR[j], 0.5 * sDq[2 * n1 + i][v], ae);
      sGc[v][t] = sM[4][t] * fma(sM[0][t], ax, sM[2][t] * ae);
      sGc[3 + v][t] = sM[4][t] * fma(sM[1][t], ax, sM[3][t] * ae);
    }
  }
  for (int t = tid; t < FP; t += nt) {
    const int f = t / n1, k = t - f * n1;
    const bool plus = (f == 1 || f == 2), eta = (f == 0 || f == 2);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) s = fma(plus ? slp[m] : slm[m], sGb[c][eta ? m * n1 + k : k * n1 + m], s);
      const double nc = c < 3 ? sS[t][0] : sS[t][1];
      const double other = sBc[f] ? s : sGf[t][c];   // a boundary mirrors the element
      sGf[t][c] = fma(sS[t][3] * nc, sDq[t][c % 3], 0.5 * (s + other));
    }
  }
  __syncthreads();

  double* Db = Dout + (size_t)e * n * n;
  for (int c0 = 0; c0 < 3 * N; c0 += C) {
    // (A) tangents of the total contravariant fluxes at the solution points
    for (int t = tid; t < C * N; t += nt) {
      const int cc = t / N, pt = t - cc * N, col = c0 + cc;
      if (col >= 3 * N) continue;
      const int w = col / N, cp = col - w * N, ci = cp % n1, cj = cp / n1;
      const int i = pt % n1, j = pt / n1;
      // d(corrected reference derivative)/dq: D plus the DG correction of
      // d(q_com - q^-) = kappa dq^- on the two faces of each line
      const double dax =
          (cj == j) ? sD[i][ci] + sgL[i] * sKap[3][w] * slm[ci] + sgR[i] * sKap[1][w] * slp[ci] : 0.0;
      const double dae =
          (ci == i) ? sD[j][cj] + sgL[j] * sKap[0][w] * slm[cj] + sgR[j] * sKap[2][w] * slp[cj] : 0.0;
      const double a = sM[0][pt], b = sM[1][pt], c = sM[2][pt], d = sM[3][pt], iJ = sM[4][pt];
      Dual gr[6];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        gr[v] = Dual(sGc[v][pt], v == w ? iJ * fma(a, dax, c * dae) : 0.0);
        gr[3 + v] = Dual(sGc[3 + v][pt], v == w ? iJ * fma(b, dax, d * dae) : 0.0);
      }
      const Dual u(sV[0][pt], (w == 0 && cp == pt) ? 1.0 : 0.0);
      const Dual vv(sV[1][pt], (w == 1 && cp == pt) ? 1.0 : 0.0);
      Dual fv[4], gv[4];
      viscous_flux(u, vv, gr, ph, fv, gv);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        sdF[cc][r][pt] = -fma(a, fv[r + 1].d, b * gv[r + 1].d);
        sdG[cc][r][pt] = -fma(c, fv[r + 1].d, d * gv[r + 1].d);
      }
    }
    __syncthreads();
    // (B) tangents of the face jumps: common minus extrapolated flux
    for (int t = tid; t < C * FP; t += nt) {
      const int cc = t / FP, fp = t - cc * FP, col = c0 + cc;
      if (col >= 3 * N) continue;
      const int w = col / N, cp = col - w * N, ci = cp % n1, cj = cp / n1;
      const int f = fp / n1, k = fp - f * n1;
      const bool plus = (f == 1 || f == 2), xi = (f == 1 || f == 3);
      const double* l = plus ? slp : slm;
      // own trace of the perturbed variable
      const bool on_line = xi ? (cj == k) : (ci == k);
      const double dqm = on_line ? l[xi ? ci : cj] : 0.0;
      // trace of the broken-gradient tangent along the normal line
      double dgx = 0.0, dgy = 0.0;
      for (int m = 0; m < n1; ++m) {
        const int ii = xi ? m : k, jj = xi ? k : m, p2 = jj * n1 + ii;
        const double bx = (cj == jj) ? sD[ii][ci] : 0.0;
        const double be = (ci == ii) ? sD[jj][cj] : 0.0;
        dgx = fma(l[m], sM[4][p2] * fma(sM[0][p2], bx, sM[2][p2] * be), dgx);
        dgy = fma(l[m], sM[4][p2] * fma(sM[1][p2], bx, sM[3][p2] * be), dgy);
      }
      // d(grad q_com) = gfac d(grad q^-) + lifting of d(q_com - q^-) = kappa dq^-
      // (gfac = 1/2, or 1 where the ghost side mirrors the element)
      const double wl = sS[fp][3], nx = sS[fp][0], ny = sS[fp][1], dS = sS[fp][2];
      const double kap = sKap[f][w], gfac = sBc[f] ? 1.0 : 0.5;
      Dual gr[6];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        gr[v] = Dual(sGf[fp][v], v == w ? fma(2.0 * kap * wl * nx, dqm, gfac * dgx) : 0.0);
        gr[3 + v] = Dual(sGf[fp][3 + v], v == w ? fma(2.0 * kap * wl * ny, dqm, gfac * dgy) : 0.0);
      }
      const Dual u(sQc[fp][0], w == 0 ? (1.0 + kap) * dqm : 0.0);
      const Dual vv(sQc[fp][1], w == 1 ? (1.0 + kap) * dqm : 0.0);
      Dual fv[4], gv[4];
      viscous_flux(u, vv, gr, ph, fv, gv);
      const int nr = (sBc[f] && sBc[f] != PMG_BC_FARFIELD) ? 2 : 3;   // walls: no viscous energy flux
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double dcom = r < nr ? -fma(fv[r + 1].d, nx, gv[r + 1].d * ny) * dS : 0.0;   // outward, total flux
        double loc = 0.0;
        for (int m = 0; m < n1; ++m) loc = fma(l[m], xi ? sdF[cc][r][k * n1 + m] : sdG[cc][r][m * n1 + k], loc);
        sdJ[cc][f][r][k] = (plus ? dcom : -dcom) - loc;
      }
    }
    __syncthreads();
    // (C) tangent of the residual: derivative plus correction, scaled by -1/|J|
    for (int t = tid; t < C * N; t += nt) {
      const int cc = t / N, pt = t - cc * N, col = c0 + cc;
      if (col >= 3 * N) continue;
      const int w = col / N, cp = col - w * N;
      const int i = pt % n1, j = pt / n1;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double acc = 0.0;
        for (int m = 0; m < n1; ++m) {
          acc = fma(sD[i][m], sdF[cc][r][j * n1 + m], acc);
          acc = fma(sD[j][m], sdG[cc][r][m * n1 + i], acc);
        }
        acc = fma(sgL[i], sdJ[cc][3][r][j], acc);
        acc = fma(sgR[i], sdJ[cc][1][r][j], acc);
        acc = fma(sgL[j], sdJ[cc][0][r][i], acc);
        acc = fma(sgR[j], sdJ[cc][2][r][i], acc);
        const double dR = -acc * sM[4][pt];
        Db[(size_t)((r + 1) * N + pt) * n + (w + 1) * N + cp] -= dR;   // D = ... - dR/dq
      }
    }
    __syncthreads();
  }
}

void launch_assemble_visc(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s) {
  launch_grad(c, L, q, s);
  const int* nbr = c.d_faces + 5 * c.n_faces;
#define PMG_AV(PP) \
  assemble_visc_kernel<PP><<<c.E, 256, 0, s>>>(c.E, q, L.Gb, L.met, L.face, L.fJinv, nbr, L.op, c.ph, L.Dfull)
  switch (L.P) {
    case 0: PMG_AV(0); break;
    case 1: PMG_AV(1); break;
    case 2: PMG_AV(2); break;
    case 3: PMG_AV(3); break;
    case 4: PMG_AV(4); break;
    default: PMG_AV(5); break;
  }
#undef PMG_AV
}

}  // namespace pmg
