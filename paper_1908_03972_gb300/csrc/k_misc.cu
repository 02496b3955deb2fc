// k_misc.cu -- P-level transfers (Section 3) and ESDIRK stage arithmetic
// (Section 2.4, eqs. ESDIRK_ns and ESDIRK_primitive), all FP64 and HBM-bound.
#include "pmg_internal.h"

namespace pmg {

// Restriction: out[v][e][(jc,ic)] = sum_{a,b} R[ic][a] R[jc][b] in[v][e][(b,a)]
// (tensor product of the 1D L2 projection).  Optionally also writes a copy
// (out2) and scales the result (scale = -1 turns F - S into the defect).
template <int PF, int PC>
__global__ void restrict_kernel(int E, XferTab X, const double* __restrict__ in, double* __restrict__ out,
                                double* __restrict__ out2, double scale) {
  constexpr int nf = PF + 1, nc = PC + 1, Nf = nf * nf, Nc = nc * nc;
  __shared__ double sR[nc][nf];
  if (threadIdx.x < nc * nf) sR[threadIdx.x / nf][threadIdx.x % nf] = X.R[threadIdx.x / nf][threadIdx.x % nf];
  __syncthreads();
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * Nc) return;
  int e = tid / Nc, cp = tid - e * Nc, ic = cp % nc, jc = cp / nc;
  for (int v = 0; v < 4; ++v) {
    const double* src = in + ((size_t)v * E + e) * Nf;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < nf; ++b) {
      double t = 0.0;
#pragma unroll
      for (int a = 0; a < nf; ++a) t = fma(sR[ic][a], src[b * nf + a], t);
      s = fma(sR[jc][b], t, s);
    }
    s *= scale;
    size_t o = ((size_t)v * E + e) * Nc + cp;
    out[o] = s;
    if (out2) out2[o] = s;
  }
}

// Prolongation of the coarse correction: qf += I (qc - qcb), or qf = I qc
// when qcb is null and add = 0.
template <int PF, int PC>
__global__ void prolong_kernel(int E, XferTab X, const double* __restrict__ qc, const double* __restrict__ qcb,
                               double* __restrict__ qf, int add) {
  constexpr int nf = PF + 1, nc = PC + 1, Nf = nf * nf, Nc = nc * nc;
  __shared__ double sI[nf][nc];
  if (threadIdx.x < nf * nc) sI[threadIdx.x / nc][threadIdx.x % nc] = X.I[threadIdx.x / nc][threadIdx.x % nc];
  __syncthreads();
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= E * Nf) return;
  int e = tid / Nf, fp = tid - e * Nf, i = fp % nf, j = fp / nf;
  for (int v = 0; v < 4; ++v) {
    const double* a0 = qc + ((size_t)v * E + e) * Nc;
    const double* b0 = qcb ? qcb + ((size_t)v * E + e) * Nc : nullptr;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < nc; ++b) {
      double t = 0.0;
#pragma unroll
      for (int a = 0; a < nc; ++a) {
        double c = a0[b * nc + a];
        if (b0) c -= b0[b * nc + a];
        t = fma(sI[i][a], c, t);
      }
      s = fma(sI[j][b], t, s);
    }
    size_t o = ((size_t)v * E + e) * Nf + fp;
    if (add) qf[o] += s;
    else qf[o] = s;
  }
}

#define PMG_PAIRS(M) \
  M(1, 0) M(2, 0) M(2, 1) M(3, 0) M(3, 1) M(3, 2) M(4, 0) M(4, 1) M(4, 2) M(4, 3) M(5, 0) M(5, 1) M(5, 2) M(5, 3) M(5, 4)

void launch_restrict(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                     double* out, double* out2, double scale, cudaStream_t s) {
  if (c.dim == 3) { launch_restrict3(c, Lf, Lc, X, in, out, out2, scale, s); return; }
  int total = c.E * Lc.N, threads = 64, blocks = (total + threads - 1) / threads;
#define PMG_R(A, B) \
  if (Lf.P == A && Lc.P == B) { restrict_kernel<A, B><<<blocks, threads, 0, s>>>(c.E, X, in, out, out2, scale); return; }
  PMG_PAIRS(PMG_R)
#undef PMG_R
}

static void prolong_impl(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* qc,
                         const double* qcb, double* qf, int add, cudaStream_t s) {
  if (c.dim == 3) { launch_prolong3(c, Lf, Lc, X, qc, qcb, qf, add, s); return; }
  int total = c.E * Lf.N, threads = 64, blocks = (total + threads - 1) / threads;
#define PMG_P(A, B) \
  if (Lf.P == A && Lc.P == B) { prolong_kernel<A, B><<<blocks, threads, 0, s>>>(c.E, X, qc, qcb, qf, add); return; }
  PMG_PAIRS(PMG_P)
#undef PMG_P
}

void launch_prolong_add(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* qc,
                        const double* qcb, double* qf, cudaStream_t s) {
  prolong_impl(c, Lf, Lc, X, qc, qcb, qf, 1, s);
}

void launch_prolong(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                    double* out, cudaStream_t s) {
  prolong_impl(c, Lf, Lc, X, in, nullptr, out, 0, s);
}

// ------------------------------------------------------------------ stages
__global__ void cons_kernel(size_t plane, Phys ph, const double* __restrict__ q, double* __restrict__ qc) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  double qq[4] = {q[i], q[plane + i], q[2 * plane + i], q[3 * plane + i]}, o[4];
  cons(qq, ph, o);
  for (int v = 0; v < 4; ++v) qc[v * plane + i] = o[v];
}

struct RPtrs {
  const double* p[6];
  double coef[6];
};

// src = (q_c^n + dt sum_j a_ij R^j) / (omega dt); without q_c^n (split form of
// the stage system, where q_c^n enters through q_c(q) - q_c(q^n)) only the
// R-sum part is formed.
__global__ void stage_src_kernel(size_t tot, const double* __restrict__ qcn, RPtrs R, int nr, double dt,
                                 double inv_odt, double* __restrict__ src) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  double acc = qcn ? qcn[i] : 0.0;
  for (int j = 0; j < nr; ++j) acc += dt * R.coef[j] * R.p[j][i];
  src[i] = acc * inv_odt;
}

// q_c^{n+1} = q_c^n + dt sum_i b_i R^i, then back to primitive variables.
// Formed as increments of q^n (gauge pressure p - p_ref): the new pressure is
// p^n + (gamma-1) (d(rho E) - d(rho |v|^2 / 2)), so neither rho E ~ 1/Ma^2 nor
// p is rounded on the way.
__global__ void bsum_kernel(size_t plane, Phys ph, const double* __restrict__ qn, RPtrs R, int nr, double dt,
                            double* __restrict__ q) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  double d[4];
  for (int v = 0; v < 4; ++v) {
    double acc = 0.0;
    for (int j = 0; j < nr; ++j) acc += R.coef[j] * R.p[j][v * plane + i];
    d[v] = dt * acc;
  }
  double pn = qn[i], un = qn[plane + i], vn = qn[2 * plane + i], Tn = qn[3 * plane + i];
  double rhon = (pn + ph.p_ref) / Tn;
  double rho = rhon + d[0];
  double mu = rhon * un + d[1], mv = rhon * vn + d[2];
  double u = mu / rho, w = mv / rho;
  double dke = 0.5 * (mu * u + mv * w) - 0.5 * rhon * (un * un + vn * vn);
  double p = pn + ph.gm1 * (d[3] - dke);
  q[i] = p;
  q[plane + i] = u;
  q[2 * plane + i] = w;
  q[3 * plane + i] = (p + ph.p_ref) / rho;
}

// Gauge conversion of the pressure plane: q[0..plane) += delta.
__global__ void shift_kernel(size_t plane, double delta, double* __restrict__ q) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < plane) q[i] += delta;
}

void launch_shift_pressure(size_t plane, double delta, double* q, cudaStream_t s) {
  if (delta == 0.0) return;
  shift_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(plane, delta, q);
}

void launch_cons(const Ctx& c, int N, const double* q, double* qc, cudaStream_t s) {
  size_t plane = (size_t)c.E * N;
  cons_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(plane, c.ph, q, qc);
}

void launch_stage_src(const Ctx& c, int N, const double* qcn, double* const* R, const double* a, int nr,
                      double dt, double inv_odt, double* src, cudaStream_t s) {
  RPtrs rp;
  for (int j = 0; j < 6; ++j) { rp.p[j] = j < nr ? R[j] : nullptr; rp.coef[j] = j < nr ? a[j] : 0.0; }
  size_t tot = (size_t)c.nv * c.E * N;
  stage_src_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(tot, qcn, rp, nr, dt, inv_odt, src);
}

void launch_bsum_update(const Ctx& c, int N, const double* qn, double* const* R, const double* b, int nr,
                        double dt, double* q, cudaStream_t s) {
  if (c.dim == 3) { launch_bsum_update3(c, N, qn, R, b, nr, dt, q, s); return; }
  RPtrs rp;
  for (int j = 0; j < 6; ++j) { rp.p[j] = j < nr ? R[j] : nullptr; rp.coef[j] = j < nr ? b[j] : 0.0; }
  size_t plane = (size_t)c.E * N;
  bsum_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(plane, c.ph, qn, rp, nr, dt, q);
}

// dtau_min of the CFL form (Section 2.4) on the finest level: per element
// (dx/(P+1)) / max(c + |v|) and (dx/(P+1))^2 min(rho) / mu, then the minimum
// over all elements (per-block minima, then one block).
__global__ void dtau_elem_kernel(int E, int N, int P, const double* __restrict__ q, const double* __restrict__ dx,
                                 Phys ph, double* __restrict__ partial) {
  __shared__ double red[128];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double best = 1e300;
  if (e < E) {
    const size_t plane = (size_t)E * N;
    double smax = 0.0, rmin = 1e300;
    for (int p = 0; p < N; ++p) {
      const size_t i = (size_t)e * N + p;
      const double pr = q[i] + ph.p_ref, u = q[plane + i], v = q[2 * plane + i], T = q[3 * plane + i];
      smax = fmax(smax, sqrt(ph.gamma * T) + sqrt(u * u + v * v));
      rmin = fmin(rmin, pr / T);
    }
    const double hP = dx[e] / (P + 1);
    best = hP / smax;
    if (ph.mu > 0.0) best = fmin(best, hP * hP * rmin / ph.mu);
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void min_final_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double m = 1e300;
  for (int i = threadIdx.x; i < n; i += 256) m = fmin(m, partial[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

void launch_dtau_min(const Ctx& c, double* partial, double* out, cudaStream_t s) {
  const LevelDev& L = c.lev[0];
  const int blocks = (c.E + 127) / 128;
  dtau_elem_kernel<<<blocks, 128, 0, s>>>(c.E, L.N, L.P, L.q, c.d_dx, c.ph, partial);
  min_final_kernel<<<1, 256, 0, s>>>(partial, blocks, out);
}

}  // namespace pmg
