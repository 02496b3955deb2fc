// k_fused.cu -- one element-Jacobi sweep of a coarse P-level in one launch.
//
// On the coarse levels (few points per element, 4096-16384 threads per launch)
// the separate face-flux, volume and block-apply launches are each bound by
// the latency of one thread's FP64 chain, not by throughput.  This kernel
// fuses a whole sweep q_next = q + D^-1 (F(q) - S) (Section 2.4, eq.
// smoothing_element_jacobi, on the level system of Section 3) per element:
//
//  1. own state and contravariant fluxes to shared memory;
//  2. the element's own 4 (P+1) face points: own and neighbour traces (the
//     neighbour from the input state), preconditioned Roe flux, jump against
//     the extrapolated flux polynomial.  Each face is evaluated by both of
//     its elements: twice the face arithmetic, but no grid-wide dependency;
//  3. divergence + DG correction, level-system epilogue (F - S, stage term
//     relative to q^b or q^n);
//  4. x = cs .* (D^-1 (rs .* F)) with the element's factored block, written to
//     a second state buffer (Jacobi: every element reads the old state).
//
// Every global read that does not depend on an earlier phase is issued at
// entry: the blocks and their scales as bulk asynchronous copies into shared
// memory (waited for, with a bound, before phase 3), the neighbour's line
// values, the face geometry and the reference state into registers.  On the
// coarse levels one thread's latency is the kernel's time, and each of these
// would otherwise be a separate L2 round trip.
#include "sweep_common.cuh"

namespace pmg {

template <int P>
struct FusedEPB {   // elements per CTA; a thread per face point of each element
  static constexpr int value = P == 0 ? 8 : P == 1 ? 4 : P == 2 ? 2 : 1;
};

template <int P, class W>
constexpr size_t fused_smem() {   // dynamic shared memory: blocks, row scales, column scales
  constexpr size_t EPB = FusedEPB<P>::value, n = 4 * (P + 1) * (P + 1);
  return EPB * n * n * sizeof(W) + 2 * EPB * n * sizeof(double);
}

template <int P, class W, bool DWF>
__global__ void __launch_bounds__(64, 1) fused_sweep_kernel(
    int E, const double* __restrict__ qin, double* __restrict__ qout, const double* __restrict__ met,
    const double* __restrict__ face, const int* __restrict__ nbr, OpTab op, Phys ph, PhysW phw, double inv_odt,
    const double* __restrict__ src, const double* __restrict__ S, const double* __restrict__ qref,
    const W* __restrict__ Dinv, const double* __restrict__ rs, const double* __restrict__ cs,
    double* __restrict__ werr) {
  constexpr int n1 = P + 1, N = n1 * n1, n = 4 * N, EPB = FusedEPB<P>::value, FP = 4 * n1;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) unsigned long long mbar;
  W* sDinv = reinterpret_cast<W*>(dsm);
  double* srs = reinterpret_cast<double*>(dsm + (size_t)EPB * n * n * sizeof(W));
  double* scs = srs + EPB * n;
  __shared__ double sq[EPB][4][N];
  __shared__ double sFt[EPB][4][N];
  __shared__ double sGt[EPB][4][N];
  __shared__ double sJ[EPB][4][4][n1];
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[EPB][n];
  __shared__ double sD[n1][n1], sgL[n1], sgR[n1], slm[n1], slp[n1];
  const size_t plane = (size_t)E * N;
  if (threadIdx.x == 0) {
    const int e0 = blockIdx.x * EPB, ne = min(EPB, E - e0);
    const unsigned bD = (unsigned)((size_t)ne * n * n * sizeof(W)), bS = (unsigned)(ne * n * sizeof(double));
    mbar_init(&mbar);
    mbar_arrive_expect(&mbar, bD + 2 * bS);
    bulk_g2s(sDinv, Dinv + (size_t)e0 * n * n, bD, &mbar);
    bulk_g2s(srs, rs + (size_t)e0 * n, bS, &mbar);
    bulk_g2s(scs, cs + (size_t)e0 * n, bS, &mbar);
  }
  // thread (le, t): face point t = f n1 + k of element e; phase 1 and 3 point t < N
  const int le0 = threadIdx.x / FP, t0 = threadIdx.x - le0 * FP;
  const int e_0 = blockIdx.x * EPB + le0;
  const bool act = le0 < EPB && e_0 < E;
  double nq[4][n1], gx = 0.0, gy = 0.0, gS = 0.0, qo[4] = {0.0, 0.0, 0.0, 0.0};
  int fn = 0;   // neighbour's face
  if (act) {
    const int f = t0 / n1, k = t0 - f * n1;
    const int en = __ldg(nbr + (e_0 * 4 + f) * 3 + 0);
    fn = __ldg(nbr + (e_0 * 4 + f) * 3 + 1);
    const int kn = __ldg(nbr + (e_0 * 4 + f) * 3 + 2) ? P - k : k;
    const bool etan = (fn == 0 || fn == 2);
    const double* base = qin + (size_t)en * N + (etan ? kn : kn * n1);
    const int stride = etan ? n1 : 1;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int m = 0; m < n1; ++m) nq[v][m] = __ldg(base + v * plane + m * stride);
    const double* g = face + (((size_t)e_0 * 4 + f) * n1 + k) * 3;
    gx = __ldg(g);
    gy = __ldg(g + 1);
    gS = __ldg(g + 2);
    if (qref && t0 < N) {
#pragma unroll
      for (int v = 0; v < 4; ++v) qo[v] = __ldg(qref + v * plane + (size_t)e_0 * N + t0);
    }
  }
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = op.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = op.gL[threadIdx.x];
    sgR[threadIdx.x] = op.gR[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  // phase 1: thread (le, pt) for pt < N
  {
    const int le = threadIdx.x / FP, t = threadIdx.x - le * FP;
    const int e = blockIdx.x * EPB + le;
    if (le < EPB && e < E && t < N) {
      size_t gi = (size_t)e * N + t;
      double qq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) { qq[v] = __ldg(qin + v * plane + gi); sq[le][v][t] = qq[v]; }
      double qa[4] = {qq[0] + ph.p_ref, qq[1], qq[2], qq[3]};
      double a = __ldg(met + gi), b = __ldg(met + plane + gi);
      double c = __ldg(met + 2 * plane + gi), d = __ldg(met + 3 * plane + gi);
      double f[4], g[4];
      flux_xy(qa, qq[0], ph, f, g);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sFt[le][v][t] = fma(a, f[v], b * g[v]);
        sGt[le][v][t] = fma(c, f[v], d * g[v]);
      }
    }
  }
  __syncthreads();
  // phase 2: thread (le, face point t = f * n1 + k)
  {
    const int le = threadIdx.x / FP, t = threadIdx.x - le * FP;
    const int e = blockIdx.x * EPB + le;
    if (le < EPB && e < E) {
      const int f = t / n1, k = t - f * n1;
      const bool plus = (f == 1 || f == 2), eta = (f == 0 || f == 2), xi = !eta;
      const double ref[4] = {sq[le][0][0], 0.0, 0.0, sq[le][3][0]};
      double sm[4], sp[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < n1; ++m) s = fma(plus ? slp[m] : slm[m], sq[le][v][eta ? m * n1 + k : k * n1 + m] - ref[v], s);
        sm[v] = s;
      }
      {
        const bool pn = (fn == 1 || fn == 2);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < n1; ++m) s = fma(pn ? slp[m] : slm[m], nq[v][m] - ref[v], s);
          sp[v] = s;
        }
      }
      double qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) { qm[v] = ref[v] + sm[v]; qp[v] = ref[v] + sp[v]; dq[v] = sp[v] - sm[v]; }
      const double pgm = qm[0], pgp = qp[0];
      qm[0] += ph.p_ref;
      qp[0] += ph.p_ref;
      double out[4];
      face_roe<DWF>(qm, qp, dq, pgm, pgp, gx, gy, gS, ph, phw, out);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double loc = 0.0;
#pragma unroll
        for (int m = 0; m < n1; ++m)
          loc = fma(plus ? slp[m] : slm[m], xi ? sFt[le][v][k * n1 + m] : sGt[le][v][m * n1 + k], loc);
        sJ[le][f][v][k] = (plus ? out[v] : -out[v]) - loc;
      }
    }
  }
  __syncthreads();
  const bool ok = mbar_wait0(&mbar, ph.wait_ns);
  if (!ok) *werr = 1.0;
  // phase 3: residual and level-system epilogue, thread (le, pt)
  {
    const int le = threadIdx.x / FP, t = threadIdx.x - le * FP;
    const int e = blockIdx.x * EPB + le;
    if (le < EPB && e < E && t < N) {
      const int i = t % n1, j = t / n1;
      size_t gi = (size_t)e * N + t;
      double qq[4] = {sq[le][0][t], sq[le][1][t], sq[le][2][t], sq[le][3][t]};
      double qc[4];
      if (qref) {
        double rho = (qq[0] + ph.p_ref) / qq[3], rhoo = (qo[0] + ph.p_ref) / qo[3];
        qc[0] = rho - rhoo;
        qc[1] = rho * qq[1] - rhoo * qo[1];
        qc[2] = rho * qq[2] - rhoo * qo[2];
        qc[3] = (qq[0] - qo[0]) * ph.inv_gm1 +
                0.5 * (rho * (qq[1] * qq[1] + qq[2] * qq[2]) - rhoo * (qo[1] * qo[1] + qo[2] * qo[2]));
      } else {
        double qa[4] = {qq[0] + ph.p_ref, qq[1], qq[2], qq[3]};
        cons(qa, ph, qc);
      }
      const double invJ = __ldg(met + 4 * plane + gi);
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
        double F = fma(-qc[v], inv_odt, R);
        if (src) F += src[o];
        if (S) F -= S[o];
        int row = v * N + t;
        sr[le][row] = scaled_in<W>(F, ok ? srs[le * n + row] : rs[(size_t)e * n + row]);
      }
    }
  }
  __syncthreads();
  // phase 4: block apply, thread (le, rows 4t..4t+3) for t < N
  {
    const int le = threadIdx.x / FP, t = threadIdx.x - le * FP;
    const int e = blockIdx.x * EPB + le;
    if (le < EPB && e < E && t < N) {
      Acc acc[4] = {0, 0, 0, 0};
      const W* Dm = ok ? sDinv + (size_t)le * n * n + 4 * t : Dinv + (size_t)e * n * n + 4 * t;
#pragma unroll 4
      for (int kk = 0; kk < n; ++kk) {
        Acc rk = sr[le][kk];
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = fma(blk_val(Dm[(size_t)kk * n + m]), rk, acc[m]);
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int row = 4 * t + m;
        int v = row / N, pt = row - v * N;
        double xv = scaled_out<W>(acc[m], ok ? scs[le * n + row] : cs[(size_t)e * n + row]);
        size_t o = v * plane + (size_t)e * N + pt;
        qout[o] = sq[le][v][pt] + xv;
      }
    }
  }
  if (!ok) mbar_drain0(&mbar);   // copies still in flight land before the CTA exits
}

// The same sweep in double-word arithmetic (gauge storage, the sweeps of
// PMG_FLUX_DW_SMOOTH): contravariant fluxes, face fluxes, face jumps, the
// divergence and the level-system epilogue run on the FP32 pipes (dword.cuh;
// see k_volume_dw.cu), while the traces and jumps the face flux takes are
// still formed in binary64 relative to the element's first point.
template <int P, class W>
__global__ void __launch_bounds__(64, 1) fused_sweep_dw_kernel(
    int E, const double* __restrict__ qin, double* __restrict__ qout, const double* __restrict__ met,
    const double* __restrict__ face, const int* __restrict__ nbr, OpTabW opw, OpTab op, PhysW k, double p_ref,
    double inv_odt, const double* __restrict__ S, const double* __restrict__ qref, const W* __restrict__ Dinv,
    const double* __restrict__ rs, const double* __restrict__ cs, double* __restrict__ werr) {
  constexpr int n1 = P + 1, N = n1 * n1, n = 4 * N, EPB = FusedEPB<P>::value, FP = 4 * n1;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) unsigned long long mbar;
  W* sDinv = reinterpret_cast<W*>(dsm);
  double* srs = reinterpret_cast<double*>(dsm + (size_t)EPB * n * n * sizeof(W));
  double* scs = srs + EPB * n;
  __shared__ double sq[EPB][4][N];
  __shared__ dw sFt[EPB][4][N];
  __shared__ dw sGt[EPB][4][N];
  __shared__ dw sJ[EPB][4][4][n1];
  using Acc = typename Blk<W>::acc;
  __shared__ Acc sr[EPB][n];
  __shared__ double slm[n1], slp[n1];
  __shared__ dw sD[n1][n1], sgL[n1], sgR[n1], swm[n1], swp[n1];
  const size_t plane = (size_t)E * N;
  if (threadIdx.x == 0) {
    const int e0 = blockIdx.x * EPB, ne = min(EPB, E - e0);
    const unsigned bD = (unsigned)((size_t)ne * n * n * sizeof(W)), bS = (unsigned)(ne * n * sizeof(double));
    mbar_init(&mbar);
    mbar_arrive_expect(&mbar, bD + 2 * bS);
    bulk_g2s(sDinv, Dinv + (size_t)e0 * n * n, bD, &mbar);
    bulk_g2s(srs, rs + (size_t)e0 * n, bS, &mbar);
    bulk_g2s(scs, cs + (size_t)e0 * n, bS, &mbar);
  }
  // thread (le, t): face point t = f n1 + k of element e; phases 1 and 3: point t < N
  const int le = threadIdx.x / FP, t = threadIdx.x - le * FP;
  const int e = blockIdx.x * EPB + le;
  const bool act = le < EPB && e < E;
  const bool own = act && t < N;
  const int f = t / n1, kf = t - f * n1;
  double nq[4][n1], gx = 0.0, gy = 0.0, gS = 0.0, qq[4] = {0, 0, 0, 0}, qo[4] = {0, 0, 0, 0};
  double Sv[4] = {0, 0, 0, 0}, mt[5] = {0, 0, 0, 0, 0};
  int fn = 0;   // neighbour's face
  if (act) {
    const int en = __ldg(nbr + (e * 4 + f) * 3 + 0);
    fn = __ldg(nbr + (e * 4 + f) * 3 + 1);
    const int kn = __ldg(nbr + (e * 4 + f) * 3 + 2) ? P - kf : kf;
    const bool etan = (fn == 0 || fn == 2);
    const double* base = qin + (size_t)en * N + (etan ? kn : kn * n1);
    const int stride = etan ? n1 : 1;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int m = 0; m < n1; ++m) nq[v][m] = __ldg(base + v * plane + m * stride);
    const double* g = face + (((size_t)e * 4 + f) * n1 + kf) * 3;
    gx = __ldg(g);
    gy = __ldg(g + 1);
    gS = __ldg(g + 2);
  }
  if (own) {
    const size_t gi = (size_t)e * N + t;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qq[v] = __ldg(qin + v * plane + gi);
      if (qref) qo[v] = __ldg(qref + v * plane + gi);
      if (S) Sv[v] = -__ldg(S + v * plane + gi);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) mt[c] = __ldg(met + c * plane + gi);
  }
  if (threadIdx.x < n1 * n1) sD[threadIdx.x / n1][threadIdx.x % n1] = opw.D[threadIdx.x / n1][threadIdx.x % n1];
  if (threadIdx.x < n1) {
    sgL[threadIdx.x] = opw.gL[threadIdx.x];
    sgR[threadIdx.x] = opw.gR[threadIdx.x];
    swm[threadIdx.x] = opw.lm[threadIdx.x];
    swp[threadIdx.x] = opw.lp[threadIdx.x];
    slm[threadIdx.x] = op.lm[threadIdx.x];
    slp[threadIdx.x] = op.lp[threadIdx.x];
  }
  // phase 1: own state to shared memory (binary64, for the traces) and the
  // contravariant fluxes in double-word
  dw Q[4], rho = {0.0f, 0.0f};
  if (own) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sq[le][v][t] = qq[v];
      Q[v] = dw_from_double(qq[v]);   // gauge p, u, v, T
    }
    rho = (Q[0] + k.p_ref) * rcp(Q[3]);
    const dw a = dw_from_double(mt[0]), b = dw_from_double(mt[1]);
    const dw c = dw_from_double(mt[2]), d = dw_from_double(mt[3]);
    const dw H = k.Cp * Q[3] + half(Q[1] * Q[1] + Q[2] * Q[2]);
    const dw mx = rho * Q[1], my = rho * Q[2];
    const dw fx[4] = {mx, mx * Q[1] + Q[0], mx * Q[2], mx * H};
    const dw gy4[4] = {my, my * Q[1], my * Q[2] + Q[0], my * H};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dw_acc x, y;
      x.add_prod(a, fx[v]);
      x.add_prod(b, gy4[v]);
      y.add_prod(c, fx[v]);
      y.add_prod(d, gy4[v]);
      sFt[le][v][t] = x.value();
      sGt[le][v][t] = y.value();
    }
  }
  __syncthreads();
  // phase 2: face point (f, kf): binary64 traces relative to the element's
  // first point, the double-word face flux, the jump against the extrapolated
  // flux polynomial
  if (act) {
    const bool plus = (f == 1 || f == 2), eta = (f == 0 || f == 2), xi = !eta;
    const double ref[4] = {sq[le][0][0], 0.0, 0.0, sq[le][3][0]};
    double sm[4], sp[4];
    const bool pn = (fn == 1 || fn == 2);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        a = fma(plus ? slp[m] : slm[m], sq[le][v][eta ? m * n1 + kf : kf * n1 + m] - ref[v], a);
        b = fma(pn ? slp[m] : slm[m], nq[v][m] - ref[v], b);
      }
      sm[v] = a;
      sp[v] = b;
    }
    double qm[4], qp[4], dq[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qm[v] = ref[v] + sm[v];
      qp[v] = ref[v] + sp[v];
      dq[v] = sp[v] - sm[v];
    }
    const double pgm = qm[0], pgp = qp[0];
    qm[0] += p_ref;
    qp[0] += p_ref;
    dw out[4];
    face_roe_dw(qm, qp, dq, pgm, pgp, gx, gy, gS, k, out);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      dw_acc loc;
#pragma unroll
      for (int m = 0; m < n1; ++m)
        loc.add_prod(plus ? swp[m] : swm[m], xi ? sFt[le][v][kf * n1 + m] : sGt[le][v][m * n1 + kf]);
      sJ[le][f][v][kf] = (plus ? out[v] : -out[v]) - loc.value();
    }
  }
  __syncthreads();
  const bool ok = mbar_wait0(&mbar, k.wait_ns);
  if (!ok) *werr = 1.0;
  // phase 3: divergence, DG correction and level-system epilogue
  if (own) {
    const int i = t % n1, j = t / n1;
    dw qc[4];
    if (qref) {
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
      dw_acc F;   // -acc / |J| - qc / (omega dt) - S
      F.add_prod(-acc.value(), invJ);
      F.add_prod(qc[v], nodt);
      F.add(dw_from_double(Sv[v]));
      const int row = v * N + t;
      sr[le][row] = scaled_in_dw<W>(F.value(), ok ? srs[le * n + row] : rs[(size_t)e * n + row]);
    }
  }
  __syncthreads();
  // phase 4: block apply, rows 4t..4t+3
  if (own) {
    Acc acc[4] = {0, 0, 0, 0};
    const W* Dm = ok ? sDinv + (size_t)le * n * n + 4 * t : Dinv + (size_t)e * n * n + 4 * t;
#pragma unroll 4
    for (int kk = 0; kk < n; ++kk) {
      const Acc rk = sr[le][kk];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] = fma(blk_val(Dm[(size_t)kk * n + m]), rk, acc[m]);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int row = 4 * t + m;
      const int v = row / N, pt = row - v * N;
      const double xv = scaled_out<W>(acc[m], ok ? scs[le * n + row] : cs[(size_t)e * n + row]);
      qout[v * plane + (size_t)e * N + pt] = sq[le][v][pt] + xv;
    }
  }
  if (!ok) mbar_drain0(&mbar);   // copies still in flight land before the CTA exits
}

template <int P>
static void fused_launch(const Ctx& c, const LevelDev& L, const double* qin, double* qout, double inv_odt,
                         const double* src, const double* S, const double* qref, int prec, cudaStream_t s) {
  constexpr int EPB = FusedEPB<P>::value, FP = 4 * (P + 1);
  int threads = (EPB * FP + 31) / 32 * 32;
  int blocks = (c.E + EPB - 1) / EPB;
  const int* nbr = c.d_faces + 5 * c.n_faces;
#define PMG_FUSED(WT, D)                                                                                    \
  fused_sweep_kernel<P, WT, D><<<blocks, threads, fused_smem<P, WT>(), s>>>(                                 \
      c.E, qin, qout, L.met, L.face, nbr, L.op, c.ph, c.phw, inv_odt, src, S, qref, (const WT*)L.Dinv, L.rs, \
      L.cs, c.d_scal + 1)
  const bool dwf = flux_dw_sweep(c);
  if (dwf && c.ph.p_ref != 0.0 && !src) {   // gauge storage: the double-word sweep
#define PMG_FUSED_DW(WT)                                                                         \
  fused_sweep_dw_kernel<P, WT><<<blocks, threads, fused_smem<P, WT>(), s>>>(                       \
      c.E, qin, qout, L.met, L.face, nbr, L.opw, L.op, c.phw, c.ph.p_ref, inv_odt, S, qref,        \
      (const WT*)L.Dinv, L.rs, L.cs, c.d_scal + 1)
    if (prec == PMG_PREC_FP64) PMG_FUSED_DW(double);
    else if (prec == PMG_PREC_BF16R) PMG_FUSED_DW(__nv_bfloat16);
    else PMG_FUSED_DW(float);
#undef PMG_FUSED_DW
    return;
  }
  if (prec == PMG_PREC_FP64) {
    if (dwf) PMG_FUSED(double, true);
    else PMG_FUSED(double, false);
  } else if (prec == PMG_PREC_BF16R) {
    if (dwf) PMG_FUSED(__nv_bfloat16, true);
    else PMG_FUSED(__nv_bfloat16, false);
  } else {
    if (dwf) PMG_FUSED(float, true);
    else PMG_FUSED(float, false);
  }
#undef PMG_FUSED
}

void launch_fused_sweep(const Ctx& c, const LevelDev& L, const double* qin, double* qout, double inv_odt,
                        const double* src, const double* S, const double* qref, int prec, cudaStream_t s) {
  switch (L.P) {
    case 0: fused_launch<0>(c, L, qin, qout, inv_odt, src, S, qref, prec, s); break;
    case 1: fused_launch<1>(c, L, qin, qout, inv_odt, src, S, qref, prec, s); break;
    case 2: fused_launch<2>(c, L, qin, qout, inv_odt, src, S, qref, prec, s); break;
    default: fused_launch<3>(c, L, qin, qout, inv_odt, src, S, qref, prec, s); break;
  }
}

}  // namespace pmg
