// k3_residual.cu -- FR/CPR residual on hexahedra (Section 2.3 with d = 3),
// binary64.
//
// Same two-launch structure as the quadrilateral kernels (k_residual.cu):
//  * face_flux3: one thread per face point of the face list.  It extrapolates
//    both elements' solution polynomials along the lines normal to the face
//    (the neighbour's face point through the face's orientation code),
//    evaluates the preconditioned Roe flux through the face normal once and
//    writes it with opposite signs into both elements' face slots.  Boundary
//    faces take the ghost state of their type.
//  * volume3: one thread per solution point, EPB3 elements per CTA.  The
//    contravariant fluxes F^i = f . J a^i of the element's points go to
//    shared memory; the face jumps (common flux in the reference direction
//    minus the extrapolated flux polynomial), the Lagrange derivative along
//    the three directions and the DG correction follow, then the epilogue of
//    the requested mode, a deterministic per-CTA sum of squares for the norm,
//    and with APPLY the element-Jacobi update q += cs .* D^-1 (rs .* (F - S)).
//
// Layout: states q[(v*E + e)*N + pt], v < 5, pt = (k*(P+1) + j)*(P+1) + i;
// metric planes met[c*E*N + e*N + pt], c = 3 i + n for J a^i_n, c = 9 for 1/J;
// face geometry face[((e*6 + f)*NF + fp)*4] = (unit outward normal, area);
// common fluxes Fcom[((v*E + e)*6 + f)*NF + fp], outward for element e.
#include "pmg_internal.h"
#include "physics3.cuh"

namespace pmg {

template <int P>
struct EPB3 {   // elements per CTA of the volume kernel: one or two warps per CTA
  static constexpr int value = P == 0 ? 32 : P == 1 ? 8 : P == 2 ? 2 : 1;
};

// Solution point at position m on the line normal to face f through face
// point (a, b).
template <int P>
__device__ __forceinline__ int line_pt3(int f, int a, int b, int m) {
  constexpr int n1 = P + 1;
  const int d = f >> 1;
  const int i = d == 0 ? m : a;
  const int j = d == 1 ? m : (d == 0 ? a : b);
  const int k = d == 2 ? m : b;
  return (k * n1 + j) * n1 + i;
}

// Trace of the solution polynomial at face point (a, b) of face f, minus ref.
template <int P>
__device__ __forceinline__ void line_trace3(const double* __restrict__ q, size_t plane, int e, int f, int a, int b,
                                            const double* lm, const double* lp, const double ref[5],
                                            double out[5]) {
  constexpr int n1 = P + 1, N = n1 * n1 * n1;
  const double* base = q + (size_t)e * N;
  const bool plus = f & 1;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < n1; ++m)
      s = fma(plus ? lp[m] : lm[m], __ldg(base + v * plane + line_pt3<P>(f, a, b, m)) - ref[v], s);
    out[v] = s;
  }
}

// With VISC (mu > 0) the face launch also forms the viscous common flux of
// eq. com_grad_q at q_com: the mean of both sides' broken-gradient traces
// (Gb, extrapolated along each side's normal line; a boundary mirrors the
// element) plus the BR2 lifting pen (1/|J|^- + 1/|J|^+)/4 dS n (q^+ - q^-);
// walls carry no viscous energy flux.  It writes q_com - q_own of
// (u, v, w, T) for both elements (Qj), the jumps the volume launch's
// corrected gradient takes.
template <int P, bool VISC>
__global__ void __launch_bounds__(64) face_flux3_kernel(const int* __restrict__ faces, int n_faces, int E,
                                                        const double* __restrict__ q,
                                                        const double* __restrict__ face,
                                                        double* __restrict__ Fcom, OpTab op, Phys ph,
                                                        const double* __restrict__ Gb,
                                                        const double* __restrict__ fJinv,
                                                        double* __restrict__ Qj) {
  constexpr int n1 = P + 1, N = n1 * n1 * n1, NF = n1 * n1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n_faces * NF) return;
  const int fc = tid / NF, fp = tid - fc * NF;
  const int a = fp % n1, b = fp / n1;
  const int* fr = faces + fc * 5;
  const int eL = fr[0], fL = fr[1], eR = fr[2], fR = fr[3], o = fr[4];
  const bool bnd = eR < 0;
  const size_t plane = (size_t)E * N;
  double lm[n1], lp[n1];
#pragma unroll
  for (int m = 0; m < n1; ++m) { lm[m] = op.lm[m]; lp[m] = op.lp[m]; }
  const double ref[5] = {__ldg(q + (size_t)eL * N), 0.0, 0.0, 0.0, __ldg(q + 4 * plane + (size_t)eL * N)};
  const double* g = face + (((size_t)eL * 6 + fL) * NF + fp) * 4;
  const double nrm[3] = {__ldg(g), __ldg(g + 1), __ldg(g + 2)};
  const double dS = __ldg(g + 3);
  double sm[5], sp[5];
  line_trace3<P>(q, plane, eL, fL, a, b, lm, lp, ref, sm);
  int fp2 = fp;
  if (!bnd) {
    const int s = (o & 4) ? b : a, t = (o & 4) ? a : b;
    const int a2 = (o & 1) ? P - s : s, b2 = (o & 2) ? P - t : t;
    fp2 = b2 * n1 + a2;
    line_trace3<P>(q, plane, eR, fR, a2, b2, lm, lp, ref, sp);
  } else if (fR == PMG_BC_FARFIELD) {
    sp[0] = (ph.qinf[0] - ph.p_ref) - ref[0];
    sp[1] = ph.qinf[1];
    sp[2] = ph.qinf[2];
    sp[3] = ph.qinf[3];
    sp[4] = ph.qinf[4] - ref[4];
  } else if (fR == PMG_BC_NOSLIP_WALL) {   // same p and T, velocity reversed
    sp[0] = sm[0];
    sp[4] = sm[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) sp[1 + c] = -sm[1 + c];
  } else {   // slip wall: same p and T, normal velocity reflected
    const double un = sm[1] * nrm[0] + sm[2] * nrm[1] + sm[3] * nrm[2];
    sp[0] = sm[0];
    sp[4] = sm[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) sp[1 + c] = fma(-2.0 * un, nrm[c], sm[1 + c]);
  }
  double qm[5], qp[5], dq[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qm[v] = ref[v] + sm[v];
    qp[v] = ref[v] + sp[v];
    dq[v] = sp[v] - sm[v];
  }
  const double pgm = qm[0], pgp = qp[0];
  qm[0] += ph.p_ref;
  qp[0] += ph.p_ref;
  double out[5];
  roe3_flux_jump(qm, qp, dq, pgm, pgp, nrm, dS, ph, out);
  const size_t fplane = (size_t)E * 6 * NF;
  const size_t iL = ((size_t)eL * 6 + fL) * NF + fp;
  if (VISC) {
    double gm[12], gp[12];
    const double* bL = Gb + (size_t)eL * N;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double t = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m)
        t = fma((fL & 1) ? lp[m] : lm[m], __ldg(bL + c * plane + line_pt3<P>(fL, a, b, m)), t);
      gm[c] = t;
      gp[c] = t;
    }
    double iJp = __ldg(fJinv + iL);
    const double iJm = iJp;
    if (!bnd) {
      const int a2 = fp2 % n1, b2 = fp2 / n1;
      const double* bR = Gb + (size_t)eR * N;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < n1; ++m)
          t = fma((fR & 1) ? lp[m] : lm[m], __ldg(bR + c * plane + line_pt3<P>(fR, a2, b2, m)), t);
        gp[c] = t;
      }
      iJp = __ldg(fJinv + ((size_t)eR * 6 + fR) * NF + fp2);
    }
    const double wl = 0.25 * op.pen * (iJm + iJp) * dS;
    double gc[12], fv[12];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) gc[c * 4 + k] = fma(wl * nrm[c], dq[k + 1], 0.5 * (gm[c * 4 + k] + gp[c * 4 + k]));
    const double uc[3] = {0.5 * (qm[1] + qp[1]), 0.5 * (qm[2] + qp[2]), 0.5 * (qm[3] + qp[3])};
    viscous_flux3(uc, gc, ph, fv);
    const int nr = (bnd && fR != PMG_BC_FARFIELD) ? 3 : 4;   // walls: no viscous energy flux
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < nr) out[r + 1] -= (fv[r] * nrm[0] + fv[4 + r] * nrm[1] + fv[8 + r] * nrm[2]) * dS;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Qj[k * fplane + iL] = 0.5 * dq[k + 1];
      if (!bnd) Qj[k * fplane + ((size_t)eR * 6 + fR) * NF + fp2] = -0.5 * dq[k + 1];
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) Fcom[v * fplane + iL] = out[v];
  if (!bnd) {
    const size_t iR = ((size_t)eR * 6 + fR) * NF + fp2;
#pragma unroll
    for (int v = 0; v < 5; ++v) Fcom[v * fplane + iR] = -out[v];
  }
}

// With VISC the contravariant fluxes take f_inv - f_vis: the viscous flux at
// each solution point from the corrected gradient, the reference derivatives
// of (u, v, w, T) plus the DG correction of the face jumps Qj on the two faces
// of each line through the point (eq. com_q), then the chain rule with the
// metric terms.
template <int P, class W, bool APPLY, bool VISC>
__global__ void __launch_bounds__(64) volume3_kernel(int E, const double* q, const double* __restrict__ met,
                                                     const double* __restrict__ Fcom, const double* __restrict__ Qj,
                                                     OpTab op, Phys ph,
                                                     double* __restrict__ out, int mode, double inv_odt,
                                                     const double* __restrict__ src, const double* __restrict__ S,
                                                     double* __restrict__ Sout, const double* __restrict__ Pd,
                                                     const double* __restrict__ qn, double* __restrict__ partial,
                                                     double* qw, const W* __restrict__ Dinv,
                                                     const double* __restrict__ rs, const double* __restrict__ cs) {
  constexpr int n1 = P + 1, N = n1 * n1 * n1, NF = n1 * n1, EPB = EPB3<P>::value, n = 5 * N;
  using Acc = typename Blk<W>::acc;
  __shared__ double sF[EPB][3][5][N];
  __shared__ double sJ[EPB][6][5][NF];
  __shared__ Acc sr[APPLY ? EPB : 1][APPLY ? n : 1];
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  __shared__ double sred[2];
  __shared__ double sV[VISC ? EPB : 1][4][VISC ? N : 1];   // u, v, w, T of the element
  const int le = threadIdx.x / N, pt = threadIdx.x - le * N;
  const int e = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (e < E);
  const size_t plane = (size_t)E * N;
  const size_t fplane = (size_t)E * 6 * NF;
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = op.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = op.gL[threadIdx.x];
    sgR[threadIdx.x] = op.gR[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  const size_t gi = (size_t)e * N + pt;
  double qq[5] = {0, 0, 0, 0, 0}, invJ = 0.0, rho_pt = 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) qq[v] = q[v * plane + gi];
    invJ = __ldg(met + 9 * plane + gi);
    if (VISC)
#pragma unroll
      for (int k = 0; k < 4; ++k) sV[VISC ? le : 0][k][VISC ? pt : 0] = qq[k + 1];
  }
  if (VISC) __syncthreads();
  if (active) {
    double qa[5] = {qq[0] + ph.p_ref, qq[1], qq[2], qq[3], qq[4]};
    rho_pt = qa[0] * s_rcp(qa[4]);
    double ja[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) ja[i][c] = __ldg(met + (3 * i + c) * plane + gi);
    double fv[12];
    if (VISC) {
      const int i = pt % n1, j = (pt / n1) % n1, k = pt / (n1 * n1);
      const int idx[3] = {i, j, k}, fpd[3] = {k * n1 + j, k * n1 + i, j * n1 + i};
      double g[12];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const double* V = sV[VISC ? le : 0][w];
        double dr[3] = {0.0, 0.0, 0.0};
        const double r0 = V[(k * n1 + j) * n1], r1 = V[k * n1 * n1 + i], r2 = V[j * n1 + i];
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          dr[0] = fma(sD[i][m], V[(k * n1 + j) * n1 + m] - r0, dr[0]);
          dr[1] = fma(sD[j][m], V[(k * n1 + m) * n1 + i] - r1, dr[1]);
          dr[2] = fma(sD[k][m], V[(m * n1 + j) * n1 + i] - r2, dr[2]);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dr[d] = fma(sgL[idx[d]], __ldg(Qj + w * fplane + ((size_t)e * 6 + 2 * d) * NF + fpd[d]), dr[d]);
          dr[d] = fma(sgR[idx[d]], __ldg(Qj + w * fplane + ((size_t)e * 6 + 2 * d + 1) * NF + fpd[d]), dr[d]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c * 4 + w] = invJ * (ja[0][c] * dr[0] + ja[1][c] * dr[1] + ja[2][c] * dr[2]);
      }
      const double uvw[3] = {qq[1], qq[2], qq[3]};
      viscous_flux3(uvw, g, ph, fv);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double f[5];
      flux3_n(qa, qq[0], ja[i], ph, f);
      if (VISC)
#pragma unroll
        for (int r = 0; r < 4; ++r) f[r + 1] -= ja[i][0] * fv[r] + ja[i][1] * fv[4 + r] + ja[i][2] * fv[8 + r];
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[le][i][v][pt] = f[v];
    }
  }
  __syncthreads();
  if (active) {
    for (int it = pt; it < 30 * NF; it += N) {
      const int f = it / (5 * NF), r = it - f * 5 * NF, v = r / NF, fp = r - v * NF;
      const int a = fp % n1, b = fp / n1, d = f >> 1;
      const bool plus = f & 1;
      double loc = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m) loc = fma(plus ? slp[m] : slm[m], sF[le][d][v][line_pt3<P>(f, a, b, m)], loc);
      const double com = __ldg(Fcom + v * fplane + ((size_t)e * 6 + f) * NF + fp);
      sJ[le][f][v][fp] = (plus ? com : -com) - loc;
    }
  }
  __syncthreads();
  double ssq = 0.0;
  if (active) {
    const int i = pt % n1, j = (pt / n1) % n1, k = pt / (n1 * n1);
    double qc[5];
    if (qn) {
      // q_c(q) - q_c(q_ref) with the energy through the pressure difference
      double qo[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qo[v] = __ldg(qn + v * plane + gi);
      const double rho = rho_pt, rhoo = (qo[0] + ph.p_ref) * s_rcp(qo[4]);
      qc[0] = rho - rhoo;
#pragma unroll
      for (int c = 1; c < 4; ++c) qc[c] = rho * qq[c] - rhoo * qo[c];
      qc[4] = (qq[0] - qo[0]) * ph.inv_gm1 +
              0.5 * (rho * (qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]) -
                     rhoo * (qo[1] * qo[1] + qo[2] * qo[2] + qo[3] * qo[3]));
    } else {
      qc[0] = rho_pt;
#pragma unroll
      for (int c = 1; c < 4; ++c) qc[c] = rho_pt * qq[c];
      qc[4] = rho_pt * (qq[4] * ph.inv_gm1 + 0.5 * (qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        acc = fma(sD[i][m], sF[le][0][v][(k * n1 + j) * n1 + m], acc);
        acc = fma(sD[j][m], sF[le][1][v][(k * n1 + m) * n1 + i], acc);
        acc = fma(sD[k][m], sF[le][2][v][(m * n1 + j) * n1 + i], acc);
      }
      acc = fma(sgL[i], sJ[le][0][v][k * n1 + j], acc);
      acc = fma(sgR[i], sJ[le][1][v][k * n1 + j], acc);
      acc = fma(sgL[j], sJ[le][2][v][k * n1 + i], acc);
      acc = fma(sgR[j], sJ[le][3][v][k * n1 + i], acc);
      acc = fma(sgL[k], sJ[le][4][v][j * n1 + i], acc);
      acc = fma(sgR[k], sJ[le][5][v][j * n1 + i], acc);
      const double R = -acc * invJ;
      const size_t o = v * plane + gi;
      if (mode == RES_PURE) {
        out[o] = R;
      } else if (mode == RES_FORCING) {
        const double Fraw = fma(-qc[v], inv_odt, R);
        const double pd = Pd[o];
        Sout[o] = Fraw + pd;
        out[o] = -pd;
        ssq = fma(pd, pd, ssq);
      } else {
        double F = fma(-qc[v], inv_odt, R);
        if (src) F += src[o];
        if (mode == RES_SYSTEM && S) F -= S[o];
        if (APPLY) sr[APPLY ? le : 0][APPLY ? v * N + pt : 0] = scaled_in<W>(F, rs[(size_t)e * n + v * N + pt]);
        else out[o] = F;
        if (partial) {
          const double Fw = F * ph.nw[v];
          ssq = fma(Fw, Fw, ssq);
        }
      }
    }
  }
  if (APPLY) {
    __syncthreads();
    if (active) {
      // thread (le, pt) forms the rows v N + pt (its own point) of D^-1 r;
      // the inverse is column-major, so the threads of an element read each
      // column's rows contiguously
      Acc acc[5] = {0, 0, 0, 0, 0};
      const W* Dm = Dinv + (size_t)e * n * n + pt;
      for (int kk = 0; kk < n; ++kk) {
        const Acc rk = sr[APPLY ? le : 0][APPLY ? kk : 0];
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] = fma(blk_val(__ldg(Dm + (size_t)kk * n + v * N)), rk, acc[v]);
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const size_t o = v * plane + gi;
        qw[o] = qq[v] + scaled_out<W>(acc[v], cs[(size_t)e * n + v * N + pt]);
      }
    }
  }
  if (partial) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ssq += __shfl_down_sync(0xffffffffu, ssq, off);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = ssq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += sred[w];
      partial[blockIdx.x] = s;
    }
  }
}

template <int P>
static int threads3() { return (EPB3<P>::value * (P + 1) * (P + 1) * (P + 1) + 31) / 32 * 32; }

int residual_blocks_for3(int P, int E) {
  int epb;
  switch (P) {
    case 0: epb = EPB3<0>::value; break;
    case 1: epb = EPB3<1>::value; break;
    case 2: epb = EPB3<2>::value; break;
    default: epb = EPB3<3>::value; break;
  }
  return (E + epb - 1) / epb;
}

// Broken gradient of (u, v, w, T) at every solution point of hexahedra:
// Gb[(c*4 + k) * E N + e N + pt], c = x, y, z, by the Lagrange derivative
// along the three lines through the point (of the differences to each line's
// first value: the derivative matrix annihilates constants, which keeps
// T ~ 1/Ma^2 out of the rounding) and the chain rule with J a^i / |J|.
template <int P>
__global__ void __launch_bounds__(128) grad3_kernel(int E, const double* __restrict__ q,
                                                    const double* __restrict__ met, OpTab op,
                                                    double* __restrict__ Gb) {
  constexpr int n1 = P + 1, N = n1 * n1 * n1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * N) return;
  const int e = tid / N, pt = tid - e * N, i = pt % n1, j = (pt / n1) % n1, k = pt / (n1 * n1);
  const size_t plane = (size_t)E * N;
  double ja[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 3; ++c) ja[d][c] = __ldg(met + (3 * d + c) * plane + tid);
  const double iJ = __ldg(met + 9 * plane + tid);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const double* V = q + (w + 1) * plane + (size_t)e * N;
    const double r0 = __ldg(V + (k * n1 + j) * n1), r1 = __ldg(V + k * n1 * n1 + i), r2 = __ldg(V + j * n1 + i);
    double dr[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      dr[0] = fma(op.D[i][m], __ldg(V + (k * n1 + j) * n1 + m) - r0, dr[0]);
      dr[1] = fma(op.D[j][m], __ldg(V + (k * n1 + m) * n1 + i) - r1, dr[1]);
      dr[2] = fma(op.D[k][m], __ldg(V + (m * n1 + j) * n1 + i) - r2, dr[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Gb[(c * 4 + w) * plane + tid] = iJ * (ja[0][c] * dr[0] + ja[1][c] * dr[1] + ja[2][c] * dr[2]);
  }
}

void launch_grad3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s) {
  const int total = c.E * L.N, threads = 128, blocks = (total + threads - 1) / threads;
#define PMG_G3(PP) grad3_kernel<PP><<<blocks, threads, 0, s>>>(c.E, q, L.met, L.op, L.Gb)
  switch (L.P) {
    case 0: PMG_G3(0); break;
    case 1: PMG_G3(1); break;
    case 2: PMG_G3(2); break;
    default: PMG_G3(3); break;
  }
#undef PMG_G3
}

void launch_face_flux3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s) {
  const int total = c.n_faces * L.NF, threads = 64, blocks = (total + threads - 1) / threads;
  const bool visc = c.ph.mu > 0.0;
  if (visc) launch_grad3(c, L, q, s);
#define PMG_F3(PP)                                                                                                \
  if (visc)                                                                                                       \
    face_flux3_kernel<PP, true><<<blocks, threads, 0, s>>>(c.d_faces, c.n_faces, c.E, q, L.face, L.Fcom, L.op,   \
                                                           c.ph, L.Gb, L.fJinv, L.Qj);                           \
  else                                                                                                            \
    face_flux3_kernel<PP, false><<<blocks, threads, 0, s>>>(c.d_faces, c.n_faces, c.E, q, L.face, L.Fcom, L.op,  \
                                                            c.ph, nullptr, nullptr, nullptr)
  switch (L.P) {
    case 0: PMG_F3(0); break;
    case 1: PMG_F3(1); break;
    case 2: PMG_F3(2); break;
    default: PMG_F3(3); break;
  }
#undef PMG_F3
}

void launch_volume3(const Ctx& c, const LevelDev& L, const double* q, double* out, ResMode mode, double inv_odt,
                    const double* src, const double* S, double* Sout, const double* Pd, double* partial,
                    cudaStream_t s, const double* qn) {
  const int blocks = residual_blocks_for3(L.P, c.E);
  const bool visc = c.ph.mu > 0.0;
#define PMG_V3(PP)                                                                                               \
  if (visc)                                                                                                      \
    volume3_kernel<PP, double, false, true><<<blocks, threads3<PP>(), 0, s>>>(                                  \
        c.E, q, L.met, L.Fcom, L.Qj, L.op, c.ph, out, (int)mode, inv_odt, src, S, Sout, Pd, qn, partial, nullptr, \
        nullptr, nullptr, nullptr);                                                                              \
  else                                                                                                           \
    volume3_kernel<PP, double, false, false><<<blocks, threads3<PP>(), 0, s>>>(                                 \
        c.E, q, L.met, L.Fcom, nullptr, L.op, c.ph, out, (int)mode, inv_odt, src, S, Sout, Pd, qn, partial,      \
        nullptr, nullptr, nullptr, nullptr)
  switch (L.P) {
    case 0: PMG_V3(0); break;
    case 1: PMG_V3(1); break;
    case 2: PMG_V3(2); break;
    default: PMG_V3(3); break;
  }
#undef PMG_V3
}

template <class W>
static void volume_apply3_dispatch(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                                   const double* S, const double* qn, cudaStream_t s) {
  const int blocks = residual_blocks_for3(L.P, c.E);
  const W* Dinv = (const W*)L.Dinv;
  const bool visc = c.ph.mu > 0.0;
#define PMG_VA3(PP)                                                                                             \
  if (visc)                                                                                                     \
    volume3_kernel<PP, W, true, true><<<blocks, threads3<PP>(), 0, s>>>(                                       \
        c.E, q, L.met, L.Fcom, L.Qj, L.op, c.ph, nullptr, (int)RES_SYSTEM, inv_odt, src, S, nullptr, nullptr, qn, \
        nullptr, q, Dinv, L.rs, L.cs);                                                                          \
  else                                                                                                          \
    volume3_kernel<PP, W, true, false><<<blocks, threads3<PP>(), 0, s>>>(                                      \
        c.E, q, L.met, L.Fcom, nullptr, L.op, c.ph, nullptr, (int)RES_SYSTEM, inv_odt, src, S, nullptr, nullptr, \
        qn, nullptr, q, Dinv, L.rs, L.cs)
  switch (L.P) {
    case 0: PMG_VA3(0); break;
    case 1: PMG_VA3(1); break;
    case 2: PMG_VA3(2); break;
    default: PMG_VA3(3); break;
  }
#undef PMG_VA3
}

void launch_volume_apply3(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                          const double* S, const double* qn, int prec, cudaStream_t s) {
  if (prec == PMG_PREC_FP64) volume_apply3_dispatch<double>(c, L, q, inv_odt, src, S, qn, s);
  else if (prec == PMG_PREC_BF16R) volume_apply3_dispatch<__nv_bfloat16>(c, L, q, inv_odt, src, S, qn, s);
  else volume_apply3_dispatch<float>(c, L, q, inv_odt, src, S, qn, s);
}

}  // namespace pmg
