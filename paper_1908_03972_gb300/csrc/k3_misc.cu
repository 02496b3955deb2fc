// k3_misc.cu -- P-level transfers (Section 3) and ESDIRK stage arithmetic
// (Section 2.4) on hexahedra, FP64.
#include "pmg_internal.h"
#include "physics3.cuh"

namespace pmg {

// Restriction: out[v][e][(kc,jc,ic)] = sum R[ic][a] R[jc][b] R[kc][c] in[v][e][(c,b,a)],
// the tensor product of the 1D L2 projection; optional copy and scale as in 2D.
template <int PF, int PC>
__global__ void restrict3_kernel(int E, XferTab X, const double* __restrict__ in, double* __restrict__ out,
                                 double* __restrict__ out2, double scale) {
  constexpr int nf = PF + 1, nc = PC + 1, Nf = nf * nf * nf, Nc = nc * nc * nc;
  __shared__ double sR[nc][nf];
  if (threadIdx.x < nc * nf) sR[threadIdx.x / nf][threadIdx.x % nf] = X.R[threadIdx.x / nf][threadIdx.x % nf];
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * Nc) return;
  const int e = tid / Nc, cp = tid - e * Nc, ic = cp % nc, jc = (cp / nc) % nc, kc = cp / (nc * nc);
  for (int v = 0; v < 5; ++v) {
    const double* src = in + ((size_t)v * E + e) * Nf;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < nf; ++c) {
      double t2 = 0.0;
#pragma unroll
      for (int b = 0; b < nf; ++b) {
        double t1 = 0.0;
#pragma unroll
        for (int a = 0; a < nf; ++a) t1 = fma(sR[ic][a], src[(c * nf + b) * nf + a], t1);
        t2 = fma(sR[jc][b], t1, t2);
      }
      s = fma(sR[kc][c], t2, s);
    }
    s *= scale;
    const size_t o = ((size_t)v * E + e) * Nc + cp;
    out[o] = s;
    if (out2) out2[o] = s;
  }
}

// Prolongation: qf += I (qc - qcb), or qf = I qc (add = 0, qcb null).
template <int PF, int PC>
__global__ void prolong3_kernel(int E, XferTab X, const double* __restrict__ qc, const double* __restrict__ qcb,
                                double* __restrict__ qf, int add) {
  constexpr int nf = PF + 1, nc = PC + 1, Nf = nf * nf * nf, Nc = nc * nc * nc;
  __shared__ double sI[nf][nc];
  if (threadIdx.x < nf * nc) sI[threadIdx.x / nc][threadIdx.x % nc] = X.I[threadIdx.x / nc][threadIdx.x % nc];
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * Nf) return;
  const int e = tid / Nf, fp = tid - e * Nf, i = fp % nf, j = (fp / nf) % nf, k = fp / (nf * nf);
  for (int v = 0; v < 5; ++v) {
    const double* a0 = qc + ((size_t)v * E + e) * Nc;
    const double* b0 = qcb ? qcb + ((size_t)v * E + e) * Nc : nullptr;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < nc; ++c) {
      double t2 = 0.0;
#pragma unroll
      for (int b = 0; b < nc; ++b) {
        double t1 = 0.0;
#pragma unroll
        for (int a = 0; a < nc; ++a) {
          double val = a0[(c * nc + b) * nc + a];
          if (b0) val -= b0[(c * nc + b) * nc + a];
          t1 = fma(sI[i][a], val, t1);
        }
        t2 = fma(sI[j][b], t1, t2);
      }
      s = fma(sI[k][c], t2, s);
    }
    const size_t o = ((size_t)v * E + e) * Nf + fp;
    if (add) qf[o] += s;
    else qf[o] = s;
  }
}

#define PMG_PAIRS3(M) M(1, 0) M(2, 0) M(2, 1) M(3, 0) M(3, 1) M(3, 2)

void launch_restrict3(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                      double* out, double* out2, double scale, cudaStream_t s) {
  const int total = c.E * Lc.N, threads = 64, blocks = (total + threads - 1) / threads;
#define PMG_R3(A, B)                                                                               \
  if (Lf.P == A && Lc.P == B) {                                                                    \
    restrict3_kernel<A, B><<<blocks, threads, 0, s>>>(c.E, X, in, out, out2, scale);               \
    return;                                                                                        \
  }
  PMG_PAIRS3(PMG_R3)
#undef PMG_R3
}

void launch_prolong3(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* qc,
                     const double* qcb, double* qf, int add, cudaStream_t s) {
  const int total = c.E * Lf.N, threads = 64, blocks = (total + threads - 1) / threads;
#define PMG_P3(A, B)                                                                               \
  if (Lf.P == A && Lc.P == B) {                                                                    \
    prolong3_kernel<A, B><<<blocks, threads, 0, s>>>(c.E, X, qc, qcb, qf, add);                    \
    return;                                                                                        \
  }
  PMG_PAIRS3(PMG_P3)
#undef PMG_P3
}

// q_c^{n+1} = q_c^n + dt sum_i b_i R^i back to primitive variables, formed as
// increments of q^n (gauge pressure), as in 2D.
struct RPtrs3 {
  const double* p[6];
  double coef[6];
};

__global__ void bsum3_kernel(size_t plane, Phys ph, const double* __restrict__ qn, RPtrs3 R, int nr, double dt,
                             double* __restrict__ q) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  double d[5];
  for (int v = 0; v < 5; ++v) {
    double acc = 0.0;
    for (int j = 0; j < nr; ++j) acc += R.coef[j] * R.p[j][v * plane + i];
    d[v] = dt * acc;
  }
  const double pn = qn[i], Tn = qn[4 * plane + i];
  const double vn[3] = {qn[plane + i], qn[2 * plane + i], qn[3 * plane + i]};
  const double rhon = (pn + ph.p_ref) / Tn;
  const double rho = rhon + d[0];
  double vel[3], ke_new = 0.0, ke_old = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double m = rhon * vn[c] + d[1 + c];
    vel[c] = m / rho;
    ke_new += m * vel[c];
    ke_old += rhon * vn[c] * vn[c];
  }
  const double p = pn + ph.gm1 * (d[4] - 0.5 * (ke_new - ke_old));
  q[i] = p;
  for (int c = 0; c < 3; ++c) q[(1 + c) * plane + i] = vel[c];
  q[4 * plane + i] = (p + ph.p_ref) / rho;
}

void launch_bsum_update3(const Ctx& c, int N, const double* qn, double* const* R, const double* b, int nr,
                         double dt, double* q, cudaStream_t s) {
  RPtrs3 rp;
  for (int j = 0; j < 6; ++j) { rp.p[j] = j < nr ? R[j] : nullptr; rp.coef[j] = j < nr ? b[j] : 0.0; }
  const size_t plane = (size_t)c.E * N;
  bsum3_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(plane, c.ph, qn, rp, nr, dt, q);
}

}  // namespace pmg
