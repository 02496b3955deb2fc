// k_residual.cu -- FR/CPR residual on the GPU (Section 2.3).
//
// Two launches per evaluation:
//  * face_flux: one thread per face flux point.  It extrapolates both
//    neighbouring solution polynomials along the line normal to the face,
//    evaluates the preconditioned Roe flux once and writes it, with opposite
//    signs, into both elements' face slots (no atomics, exact conservation).
//    On a boundary face the outer state is the ghost state of the boundary
//    type (physics.cuh ghost_state), formed here relative to the reference.
//  * volume: one thread per solution point, several elements per CTA.
//    Contravariant fluxes go to shared memory; the Lagrange derivative, the
//    face jumps (common minus extrapolated flux polynomial) and the DG
//    correction are applied there, followed by the epilogue of the requested
//    mode (pure R, level system residual, FAS forcing) and an optional
//    deterministic per-CTA sum of squares for the residual norm.
//
// In binary64 both kernels are bound by FP64 issue on GB300 (about 1.2
// TFLOP/s).  The face kernel's double-word variant (face_roe<true>, the
// element-Jacobi sweeps) runs the Roe flux on the FP32 pipes; the sweeps'
// residual-and-update in double-word is k_volume_dw.cu.
//
// Viscous terms (mu > 0, Section 2.1 fluxes, Section 2.3 common viscous flux):
// a gradient launch (k_viscous.cu) first forms the broken gradients of
// (u, v, T) at the solution points.  The face launch extrapolates them from
// both sides, adds the BR2 liftings of the jump to form the common gradient of
// eq. com_grad_q, evaluates the viscous flux at q_com (eq. com_q) and
// subtracts it from the Roe flux; it also stores q_com - q_own for both
// elements.  The volume launch forms the corrected gradient at each solution
// point (derivative plus DG correction of those jumps) and subtracts the
// viscous flux from the inviscid one before the divergence.
#include "sweep_common.cuh"

namespace pmg {

// Trace of the solution polynomial along the line through face point k of
// face f, extrapolated from the line's solution points minus a reference
// value ref[v] (the weights sum to one, so trace = ref + returned value).
// Subtracting a common reference before the sum keeps the rounding of
// p ~ T ~ 1/Ma^2 out of the jumps p+ - p-, T+ - T- that the preconditioned
// dissipation amplifies.
template <int P>
__device__ __forceinline__ void line_trace(const double* __restrict__ q, size_t plane, int e, int f, int k,
                                           const double* lm, const double* lp, const double ref[4],
                                           double out[4]) {
  constexpr int n1 = P + 1, N = n1 * n1;
  const bool plus = (f == 1 || f == 2);
  const bool eta = (f == 0 || f == 2);
  const double* base = q + (size_t)e * N + (eta ? k : k * n1);
  const int stride = eta ? n1 : 1;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < n1; ++m) s = fma(plus ? lp[m] : lm[m], __ldg(base + v * plane + m * stride) - ref[v], s);
    out[v] = s;
  }
}

// Trace of the six broken-gradient planes of element e at face point (f, k).
template <int P>
__device__ __forceinline__ void grad_trace(const double* __restrict__ Gb, size_t plane, int e, int f, int k,
                                           const double* lm, const double* lp, double out[6]) {
  constexpr int n1 = P + 1, N = n1 * n1;
  const bool plus = (f == 1 || f == 2);
  const bool eta = (f == 0 || f == 2);
  const double* base = Gb + (size_t)e * N + (eta ? k : k * n1);
  const int stride = eta ? n1 : 1;
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < n1; ++m) s = fma(plus ? lp[m] : lm[m], __ldg(base + v * plane + m * stride), s);
    out[v] = s;
  }
}

template <int P, bool VISC, bool DWF>
__global__ void __launch_bounds__(256) face_flux_kernel(const int* __restrict__ faces, int n_faces, int E,
                                                        const double* __restrict__ q,
                                                        const double* __restrict__ face,
                                                        double* __restrict__ Fcom, OpTab op, Phys ph, PhysW phw,
                                                        const double* __restrict__ Gb,
                                                        const double* __restrict__ fJinv,
                                                        double* __restrict__ Qj) {
  constexpr int n1 = P + 1, N = n1 * n1;
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n_faces * n1) return;
  int fc = tid / n1, k = tid - fc * n1;
  const int* fr = faces + fc * 5;
  int eL = fr[0], fL = fr[1], eR = fr[2], fR = fr[3], rev = fr[4];
  int kR = rev ? P - k : k;
  size_t plane = (size_t)E * N;
  double lm[n1], lp[n1];
#pragma unroll
  for (int m = 0; m < n1; ++m) { lm[m] = op.lm[m]; lp[m] = op.lp[m]; }
  // reference: (gauge) pressure and temperature at the left element's first solution point
  double ref[4] = {__ldg(q + (size_t)eL * N), 0.0, 0.0, __ldg(q + 3 * plane + (size_t)eL * N)};
  const double* g = face + (((size_t)eL * 4 + fL) * n1 + k) * 3;
  const double nx = __ldg(g), ny = __ldg(g + 1), dS = __ldg(g + 2);
  const bool bnd = eR < 0;   // boundary face: fR holds the boundary type
  double sm[4], sp[4];
  line_trace<P>(q, plane, eL, fL, k, lm, lp, ref, sm);
  if (!bnd) {
    line_trace<P>(q, plane, eR, fR, kR, lm, lp, ref, sp);
  } else if (fR == PMG_BC_FARFIELD) {   // ghost = free stream, relative to the reference
    sp[0] = (ph.qinf[0] - ph.p_ref) - ref[0];
    sp[1] = ph.qinf[1];
    sp[2] = ph.qinf[2];
    sp[3] = ph.qinf[3] - ref[3];
  } else {   // walls: same p and T, velocity reflected (slip) or reversed (no-slip)
    sp[0] = sm[0];
    sp[3] = sm[3];
    if (fR == PMG_BC_NOSLIP_WALL) {
      sp[1] = -sm[1];
      sp[2] = -sm[2];
    } else {
      const double un = fma(sm[1], nx, sm[2] * ny);
      sp[1] = fma(-2.0 * un, nx, sm[1]);
      sp[2] = fma(-2.0 * un, ny, sm[2]);
    }
  }
  double qm[4], qp[4], dq[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qm[v] = ref[v] + sm[v];
    qp[v] = ref[v] + sp[v];
    dq[v] = sp[v] - sm[v];
  }
  const double pgm = qm[0], pgp = qp[0];   // gauge pressures for the momentum fluxes
  qm[0] += ph.p_ref;   // absolute pressure for the averaged state and rho
  qp[0] += ph.p_ref;
  double out[4];
  face_roe<DWF>(qm, qp, dq, pgm, pgp, nx, ny, dS, ph, phw, out);
  const size_t fplane = (size_t)E * 4 * n1;
  const size_t iL = ((size_t)eL * 4 + fL) * n1 + k;
  const size_t iR = bnd ? iL : ((size_t)eR * 4 + fR) * n1 + kR;
  if (VISC) {
    // common gradient: mean of the two broken-gradient traces plus the BR2
    // liftings r^- + r^+ = pen (q_com - q^-) (1/|J|^- + 1/|J|^+) n dS, with
    // q_com - q^- = dq / 2.  A boundary face mirrors the element (its
    // gradient trace and |J|): the one-sided BR2 gradient.
    double gm[6], gp[6], gc[6];
    grad_trace<P>(Gb, plane, eL, fL, k, lm, lp, gm);
    if (!bnd) {
      grad_trace<P>(Gb, plane, eR, fR, kR, lm, lp, gp);
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) gp[c] = gm[c];
    }
    const double wl = 0.25 * op.pen * (__ldg(fJinv + iL) + __ldg(fJinv + iR)) * dS;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      gc[v] = fma(wl * nx, dq[v + 1], 0.5 * (gm[v] + gp[v]));
      gc[3 + v] = fma(wl * ny, dq[v + 1], 0.5 * (gm[3 + v] + gp[3 + v]));
    }
    double fv[4], gv[4];
    viscous_flux(0.5 * (qm[1] + qp[1]), 0.5 * (qm[2] + qp[2]), gc, ph, fv, gv);
    const int nv = (bnd && fR != PMG_BC_FARFIELD) ? 3 : 4;   // walls: no viscous energy flux
#pragma unroll
    for (int v = 1; v < 4; ++v)
      if (v < nv) out[v] -= fma(fv[v], nx, gv[v] * ny) * dS;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Qj[v * fplane + iL] = 0.5 * dq[v + 1];
      if (!bnd) Qj[v * fplane + iR] = -0.5 * dq[v + 1];
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    Fcom[v * fplane + iL] = out[v];
    if (!bnd) Fcom[v * fplane + iR] = -out[v];
  }
}

// APPLY: after forming the level-system residual F of its elements, each CTA
// also performs the element-Jacobi update q += cs .* (D^-1 (rs .* F)) in
// place (eq. smoothing_element_jacobi).  That is safe within one launch: the
// face fluxes were formed from the old state by the preceding face launch,
// and a CTA reads and writes only its own elements' states.  The update's
// inputs are prefetched at entry (VolPrefetch, sweep_common.cuh).
template <int P, class W, bool APPLY, bool VISC>
__global__ void __launch_bounds__(256, 1) volume_kernel(int E, const double* q,
                                                     const double* __restrict__ met,
                                                     const double* __restrict__ Fcom, OpTab op, Phys ph,
                                                     double* __restrict__ out, int mode, double inv_odt,
                                                     const double* __restrict__ src,
                                                     const double* __restrict__ S, double* __restrict__ Sout,
                                                     const double* __restrict__ Pd,
                                                     const double* __restrict__ qn,
                                                     double* __restrict__ partial, double* qw,
                                                     const W* __restrict__ Dinv, const double* __restrict__ rs,
                                                     const double* __restrict__ cs,
                                                     const double* __restrict__ Qj,
                                                     double* __restrict__ werr) {
  constexpr int n1 = P + 1, N = n1 * n1, EPB = ElemsPerBlock<P>::value, n = 4 * N;
  using PF = VolPrefetch<P, W>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) unsigned long long mbar[2];   // 0: face fluxes, 1: blocks and scales
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[APPLY ? EPB : 1][APPLY ? n : 1];
  __shared__ double sV[VISC ? EPB : 1][3][VISC ? N : 1];   // (u, v, T) for the gradients
  __shared__ double sFt[EPB][4][N];
  __shared__ double sGt[EPB][4][N];
  __shared__ double sJ[EPB][4][4][n1];   // [face][var][k]
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  __shared__ double sred[256 / 32];

  const int le = threadIdx.x / N, pt = threadIdx.x - le * N;
  const int e = blockIdx.x * EPB + le;
  const bool active = (le < EPB) && (e < E);
  const size_t plane = (size_t)E * N;
  const size_t fplane = (size_t)E * 4 * n1;
  W* sDinv = reinterpret_cast<W*>(dsm);
  double* srs = reinterpret_cast<double*>(dsm + PF::dinv_bytes);
  double* scs = srs + EPB * n;
  double* sFc = scs + EPB * n;   // [v][local element][face][k]
  if (APPLY && threadIdx.x == 0) {
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
  // reference and forcing states of the epilogue, loaded up front
  double qo[4] = {0, 0, 0, 0}, srcv[4] = {0, 0, 0, 0}, Sv[4] = {0, 0, 0, 0};
  if (APPLY && active) {
    const size_t g0 = (size_t)e * N + pt;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (qn) qo[v] = __ldg(qn + v * plane + g0);
      if (src) srcv[v] = __ldg(src + v * plane + g0);
      if (S) Sv[v] = __ldg(S + v * plane + g0);
    }
  }
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = op.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = op.gL[threadIdx.x];
    sgR[threadIdx.x] = op.gR[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }

  double qq[4] = {0, 0, 0, 0}, invJ = 0.0, rho_pt = 0.0;
  size_t gi = (size_t)e * N + pt;
  if (VISC) {
    if (active) {
#pragma unroll
      for (int v = 1; v < 4; ++v) sV[VISC ? le : 0][v - 1][VISC ? pt : 0] = q[v * plane + gi];
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < 4; ++v) qq[v] = q[v * plane + gi];
    double a = __ldg(met + gi), b = __ldg(met + plane + gi);
    double c = __ldg(met + 2 * plane + gi), d = __ldg(met + 3 * plane + gi);
    invJ = __ldg(met + 4 * plane + gi);
    double qa[4] = {qq[0] + ph.p_ref, qq[1], qq[2], qq[3]};   // absolute pressure
    rho_pt = qa[0] * s_rcp(qa[3]);
    double f[4], g[4];
    flux_xy_rho(qa, qq[0], rho_pt, ph, f, g);
    if (VISC) {
      // corrected gradient: reference derivatives plus the DG correction of
      // the jumps q_com - q_own at the four faces' points on this point's lines
      const int i = pt % n1, j = pt / n1;
      const double* Qe = Qj + (size_t)e * 4 * n1;
      double gr[6], fv[4], gv[4];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        double ax = 0.0, ae = 0.0;
#pragma unroll
        for (int m = 0; m < n1; ++m) {   // differences to the line's first value
          ax = fma(sD[i][m], sV[VISC ? le : 0][v][VISC ? j * n1 + m : 0] - sV[VISC ? le : 0][v][VISC ? j * n1 : 0], ax);
          ae = fma(sD[j][m], sV[VISC ? le : 0][v][VISC ? m * n1 + i : 0] - sV[VISC ? le : 0][v][VISC ? i : 0], ae);
        }
        const double* Qv = Qe + v * fplane;
        ax = fma(sgL[i], __ldg(Qv + 3 * n1 + j), ax);
        ax = fma(sgR[i], __ldg(Qv + 1 * n1 + j), ax);
        ae = fma(sgL[j], __ldg(Qv + 0 * n1 + i), ae);
        ae = fma(sgR[j], __ldg(Qv + 2 * n1 + i), ae);
        gr[v] = invJ * fma(a, ax, c * ae);
        gr[3 + v] = invJ * fma(b, ax, d * ae);
      }
      viscous_flux(qq[1], qq[2], gr, ph, fv, gv);
#pragma unroll
      for (int v = 1; v < 4; ++v) { f[v] -= fv[v]; g[v] -= gv[v]; }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sFt[le][v][pt] = fma(a, f[v], b * g[v]);
      sGt[le][v][pt] = fma(c, f[v], d * g[v]);
    }
  }
  __syncthreads();
  const bool okF = APPLY ? mbar_wait0(&mbar[0], ph.wait_ns) : true;
  if (!okF) *werr = 1.0;
  if (active) {
    // face jumps: common (reference-direction) minus extrapolated flux polynomial
    for (int it = pt; it < 16 * n1; it += N) {
      int f = it / (4 * n1), r = it - f * 4 * n1, v = r / n1, k = r - v * n1;
      const bool xi = (f == 1 || f == 3);
      const bool plus = (f == 1 || f == 2);
      double loc = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        double fv = xi ? sFt[le][v][k * n1 + m] : sGt[le][v][m * n1 + k];
        loc = fma(plus ? slp[m] : slm[m], fv, loc);
      }
      double com = (APPLY && okF) ? sFc[((v * EPB + le) * 4 + f) * n1 + k]
                                  : __ldg(Fcom + v * fplane + ((size_t)e * 4 + f) * n1 + k);
      sJ[le][f][v][k] = (plus ? com : -com) - loc;
    }
  }
  __syncthreads();
  const bool okS = APPLY ? mbar_wait0(&mbar[1], ph.wait_ns) : true;
  if (!okS) *werr = 1.0;
  double ssq = 0.0;
  if (active) {
    const int i = pt % n1, j = pt / n1;
    double qc[4];
    if (qn) {
      // q_c(q) - q_c(q_ref) with the energy difference taken through
      // rho E = p/(gamma-1) + rho|v|^2/2 and the gauge pressures, so that no
      // p ~ rho E ~ 1/Ma^2 is rounded (q_ref = q^n on the finest level, q^b on
      // coarser levels, where the constant q_c(q^b)/(omega dt) cancels in F - S)
      if (!APPLY) {
#pragma unroll
        for (int v = 0; v < 4; ++v) qo[v] = __ldg(qn + v * plane + gi);
      }
      double rho = rho_pt, rhoo = (qo[0] + ph.p_ref) * s_rcp(qo[3]);
      qc[0] = rho - rhoo;
      qc[1] = rho * qq[1] - rhoo * qo[1];
      qc[2] = rho * qq[2] - rhoo * qo[2];
      qc[3] = (qq[0] - qo[0]) * ph.inv_gm1 +
              0.5 * (rho * (qq[1] * qq[1] + qq[2] * qq[2]) - rhoo * (qo[1] * qo[1] + qo[2] * qo[2]));
    } else {
      qc[0] = rho_pt;
      qc[1] = rho_pt * qq[1];
      qc[2] = rho_pt * qq[2];
      qc[3] = rho_pt * (qq[3] * ph.inv_gm1 + 0.5 * (qq[1] * qq[1] + qq[2] * qq[2]));
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        acc = fma(sD[i][m], sFt[le][v][j * n1 + m], acc);
        acc = fma(sD[j][m], sGt[le][v][m * n1 + i], acc);
      }
      acc = fma(sgL[i], sJ[le][3][v][j], acc);
      acc = fma(sgR[i], sJ[le][1][v][j], acc);
      acc = fma(sgL[j], sJ[le][0][v][i], acc);
      acc = fma(sgR[j], sJ[le][2][v][i], acc);
      double R = -acc * invJ;
      size_t o = v * plane + gi;
      if (mode == RES_PURE) {
        out[o] = R;
      } else if (mode == RES_FORCING) {
        double Fraw = fma(-qc[v], inv_odt, R);
        double pd = Pd[o];
        Sout[o] = Fraw + pd;
        out[o] = -pd;
        ssq = fma(pd, pd, ssq);
      } else {
        double F = fma(-qc[v], inv_odt, R);
        if (src) F += APPLY ? srcv[v] : src[o];
        if (mode == RES_SYSTEM && S) F -= APPLY ? Sv[v] : S[o];
        if (APPLY) {
          const int row = v * N + pt;
          const double rsc = okS ? srs[le * n + row] : rs[(size_t)e * n + row];
          sr[APPLY ? le : 0][APPLY ? row : 0] = scaled_in<W>(F, rsc);
        } else {
          out[o] = F;
        }
        if (partial) {   // weighted sum of squares of the norm of eq. ser
          const double Fw = F * ph.nw[v];
          ssq = fma(Fw, Fw, ssq);
        }
      }
    }
  }
  if (APPLY) {
    __syncthreads();
    if (active) {
      // thread (le, pt) owns rows 4 pt .. 4 pt + 3 of its element's block
      // (column-major: the four rows of a column are one 16/32-byte vector)
      Acc acc[4] = {0, 0, 0, 0};
      if (PF::blocks && okS) {
        const W* Dm = sDinv + (size_t)le * n * n + 4 * pt;
#pragma unroll 8
        for (int kk = 0; kk < n; ++kk) {
          const Acc rk = sr[APPLY ? le : 0][APPLY ? kk : 0];
          Acc d[4];
          ld4(Dm + (size_t)kk * n, d);
#pragma unroll
          for (int m = 0; m < 4; ++m) acc[m] = fma(d[m], rk, acc[m]);
        }
      } else {
        const W* Dm = Dinv + (size_t)e * n * n + 4 * pt;
#pragma unroll 8
        for (int kk = 0; kk < n; ++kk) {
          const Acc rk = sr[APPLY ? le : 0][APPLY ? kk : 0];
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
        qw[o] = q[o] + scaled_out<W>(acc[m], csc);
      }
    }
  }
  if (partial) {
    // deterministic block sum of squares
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
  // copies still in flight land before the CTA exits
  if (!okF) mbar_drain0(&mbar[0]);
  if (!okS) mbar_drain0(&mbar[1]);
}

__global__ void norm_final_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += partial[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
}

// Whole warps only: threads beyond EPB * N idle (the block reduction uses
// full-warp shuffles).
int residual_threads_per_block(int P) {
  int t;
  switch (P) {
    case 0: t = ElemsPerBlock<0>::value * 1; break;
    case 1: t = ElemsPerBlock<1>::value * 4; break;
    case 2: t = ElemsPerBlock<2>::value * 9; break;
    case 3: t = ElemsPerBlock<3>::value * 16; break;
    case 4: t = ElemsPerBlock<4>::value * 25; break;
    default: t = ElemsPerBlock<5>::value * 36; break;
  }
  return (t + 31) / 32 * 32;
}

static int elems_per_block(int P) {
  switch (P) {
    case 0: return ElemsPerBlock<0>::value;
    case 1: return ElemsPerBlock<1>::value;
    case 2: return ElemsPerBlock<2>::value;
    case 3: return ElemsPerBlock<3>::value;
    case 4: return ElemsPerBlock<4>::value;
    default: return ElemsPerBlock<5>::value;
  }
}

int residual_blocks_for(int P, int E) { int epb = elems_per_block(P); return (E + epb - 1) / epb; }

void launch_face_flux(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s, bool sweep) {
  if (c.dim == 3) { launch_face_flux3(c, L, q, s); return; }
  int total = c.n_faces * L.n1;
  // one warp per CTA: latency-bound threads, spread over every SM
  int threads = 32, blocks = (total + threads - 1) / threads;
  const bool visc = c.ph.mu > 0.0, dwf = sweep ? flux_dw_sweep(c) : flux_dw(c, L);
  if (visc) launch_grad(c, L, q, s);
#define PMG_FACE_V(PP, V, D)                                                                                 \
  face_flux_kernel<PP, V, D><<<blocks, threads, 0, s>>>(c.d_faces, c.n_faces, c.E, q, L.face, L.Fcom, L.op, \
                                                        c.ph, c.phw, V ? L.Gb : nullptr,                    \
                                                        V ? L.fJinv : nullptr, V ? L.Qj : nullptr)
#define PMG_FACE(PP)                                   \
  do {                                                 \
    if (visc) {                                        \
      if (dwf) PMG_FACE_V(PP, true, true);             \
      else PMG_FACE_V(PP, true, false);                \
    } else {                                           \
      if (dwf) PMG_FACE_V(PP, false, true);            \
      else PMG_FACE_V(PP, false, false);               \
    }                                                  \
  } while (0)
  switch (L.P) {
    case 0: PMG_FACE(0); break;
    case 1: PMG_FACE(1); break;
    case 2: PMG_FACE(2); break;
    case 3: PMG_FACE(3); break;
    case 4: PMG_FACE(4); break;
    default: PMG_FACE(5); break;
  }
#undef PMG_FACE
#undef PMG_FACE_V
}

void launch_volume(const Ctx& c, const LevelDev& L, int level, const double* q, double* out, ResMode mode,
                   double inv_odt, const double* src, const double* S, double* Sout, const double* Pd,
                   double* partial, cudaStream_t s, const double* qn) {
  (void)level;
  if (c.dim == 3) { launch_volume3(c, L, q, out, mode, inv_odt, src, S, Sout, Pd, partial, s, qn); return; }
  int threads = residual_threads_per_block(L.P);
  int blocks = residual_blocks_for(L.P, c.E);
#define PMG_VOL(PP)                                                                                          \
  do {                                                                                                       \
    if (c.ph.mu > 0.0)                                                                                       \
      volume_kernel<PP, double, false, true><<<blocks, threads, 0, s>>>(                                     \
          c.E, q, L.met, L.Fcom, L.op, c.ph, out, (int)mode, inv_odt, src, S, Sout, Pd, qn, partial, nullptr, \
          nullptr, nullptr, nullptr, L.Qj, nullptr);                                                         \
    else                                                                                                     \
      volume_kernel<PP, double, false, false><<<blocks, threads, 0, s>>>(                                    \
          c.E, q, L.met, L.Fcom, L.op, c.ph, out, (int)mode, inv_odt, src, S, Sout, Pd, qn, partial, nullptr, \
          nullptr, nullptr, nullptr, nullptr, nullptr);                                                      \
  } while (0)
  switch (L.P) {
    case 0: PMG_VOL(0); break;
    case 1: PMG_VOL(1); break;
    case 2: PMG_VOL(2); break;
    case 3: PMG_VOL(3); break;
    case 4: PMG_VOL(4); break;
    default: PMG_VOL(5); break;
  }
#undef PMG_VOL
}

template <class W>
static void volume_apply_dispatch(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                                  const double* S, const double* qn, cudaStream_t s) {
  int threads = residual_threads_per_block(L.P);
  int blocks = residual_blocks_for(L.P, c.E);
  const W* Dinv = (const W*)L.Dinv;
  double* werr = c.d_scal + 1;
#define PMG_VA(PP)                                                                                             \
  do {                                                                                                         \
    const size_t sm = VolPrefetch<PP, W>::smem;                                                                \
    if (c.ph.mu > 0.0)                                                                                         \
      volume_kernel<PP, W, true, true><<<blocks, threads, sm, s>>>(c.E, q, L.met, L.Fcom, L.op, c.ph, nullptr,  \
                                                                   (int)RES_SYSTEM, inv_odt, src, S, nullptr,   \
                                                                   nullptr, qn, nullptr, q, Dinv, L.rs, L.cs,   \
                                                                   L.Qj, werr);                                 \
    else                                                                                                       \
      volume_kernel<PP, W, true, false><<<blocks, threads, sm, s>>>(c.E, q, L.met, L.Fcom, L.op, c.ph, nullptr, \
                                                                    (int)RES_SYSTEM, inv_odt, src, S, nullptr,  \
                                                                    nullptr, qn, nullptr, q, Dinv, L.rs, L.cs,  \
                                                                    nullptr, werr);                             \
  } while (0)
  switch (L.P) {
    case 0: PMG_VA(0); break;
    case 1: PMG_VA(1); break;
    case 2: PMG_VA(2); break;
    case 3: PMG_VA(3); break;
    case 4: PMG_VA(4); break;
    default: PMG_VA(5); break;
  }
#undef PMG_VA
}

// Level-system residual of the current state followed, in the same launch,
// by the element-Jacobi update of that state (after launch_face_flux).
void launch_volume_apply(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                         const double* S, const double* qn, int prec, cudaStream_t s) {
  if (c.dim == 3) { launch_volume_apply3(c, L, q, inv_odt, src, S, qn, prec, s); return; }
  if (prec == PMG_PREC_FP64) volume_apply_dispatch<double>(c, L, q, inv_odt, src, S, qn, s);
  else if (prec == PMG_PREC_BF16R) volume_apply_dispatch<__nv_bfloat16>(c, L, q, inv_odt, src, S, qn, s);
  else volume_apply_dispatch<float>(c, L, q, inv_odt, src, S, qn, s);
}

// Dynamic shared memory limits of the fused residual-and-update kernels of
// every level (their prefetch buffers can exceed the 48 KB default).
template <class W>
static cudaError_t prepare_apply(int P, bool visc) {
#define PMG_PREP(PP)                                                                                          \
  return visc ? cudaFuncSetAttribute(volume_kernel<PP, W, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)VolPrefetch<PP, W>::smem)                                            \
              : cudaFuncSetAttribute(volume_kernel<PP, W, true, false>,                                        \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)VolPrefetch<PP, W>::smem)
  switch (P) {
    case 0: PMG_PREP(0);
    case 1: PMG_PREP(1);
    case 2: PMG_PREP(2);
    case 3: PMG_PREP(3);
    case 4: PMG_PREP(4);
    default: PMG_PREP(5);
  }
#undef PMG_PREP
}

cudaError_t prepare_residual_kernels(const Ctx& c) {
  for (int l = 0; l < c.cfg.n_levels; ++l) {
    const bool visc = c.ph.mu > 0.0;
    cudaError_t e = c.cfg.block_prec == PMG_PREC_FP64    ? prepare_apply<double>(c.lev[l].P, visc)
                    : c.cfg.block_prec == PMG_PREC_BF16R ? prepare_apply<__nv_bfloat16>(c.lev[l].P, visc)
                                                         : prepare_apply<float>(c.lev[l].P, visc);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_norm_final(const double* partial, int n, double* out, cudaStream_t s) {
  norm_final_kernel<<<1, 256, 0, s>>>(partial, n, out);
}

}  // namespace pmg
