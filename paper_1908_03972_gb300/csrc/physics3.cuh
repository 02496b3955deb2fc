// physics3.cuh -- pointwise physics of the three-dimensional solver:
// primitive working variables (p, u, v, w, T), R = 1 (Sections 2.1-2.2 with
// d = 3).  Same conventions as physics.cuh: q holds the absolute pressure and
// pm is the pressure put into the momentum flux (the gauge pressure p - p_ref
// with gauge storage), templates over double and Dual.
#pragma once
#include "physics.cuh"

namespace pmg {

// Inviscid flux through the (not necessarily unit) vector n.
template <class S>
__host__ __device__ inline void flux3_n(const S q[5], const S& pm, const double n[3], const Phys& ph, S f[5]) {
  S rho = q[0] * s_rcp(q[4]);
  S H = ph.Cp * q[4] + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S mn = rho * (q[1] * n[0] + q[2] * n[1] + q[3] * n[2]);
  f[0] = mn;
  f[1] = mn * q[1] + pm * n[0];
  f[2] = mn * q[2] + pm * n[1];
  f[3] = mn * q[3] + pm * n[2];
  f[4] = mn * H;
}

// Conservative variables (rho, rho u, rho v, rho w, rho E).
template <class S>
__host__ __device__ inline void cons3(const S q[5], const Phys& ph, S qc[5]) {
  S rho = q[0] / q[4];
  qc[0] = rho;
  qc[1] = rho * q[1];
  qc[2] = rho * q[2];
  qc[3] = rho * q[3];
  qc[4] = rho * (q[4] * ph.inv_gm1 + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]));
}

template <class S>
__host__ __device__ inline S eps2_of3(const S q[5], const Phys& ph) {
  S ma2 = (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / (ph.gamma * q[4]);
  return s_min(S(1.0), s_max(S(ph.eps_min * ph.eps_min), ma2));
}

// Preconditioned Roe flux (eq. invis_com) through unit normal n times the
// face area dS, every matrix at the arithmetic mean of the primitive states.
// The closed form of the 2D flux carries over: in rotated primitive variables
// (p, u_n, u_t1, u_t2, T) the matrix K^-1 M^-1 A_n is block lower triangular
// with the acoustic block B on (p, u_n), both tangential components
// decoupled with eigenvalue u_n, and the T row coupled to (p, u_n) with
// eigenvalue u_n; the tangential part of the dissipation is |u_n| times the
// tangential velocity jump, i.e. |u_n| (dv - (dv.n) n) in Cartesian form.
template <class S>
__host__ __device__ inline void roe3_flux_jump(const S qm[5], const S qp[5], const S dq[5], const S& pmm,
                                               const S& pmp, const double n[3], double dS, const Phys& ph,
                                               S out[5]) {
  S fm[5], fp[5];
  flux3_n(qm, pmm, n, ph, fm);
  flux3_n(qp, pmp, n, ph, fp);
  const S dp = dq[0], dT = dq[4];
  const S dvel[3] = {dq[1], dq[2], dq[3]};
  const S p = qm[0] + 0.5 * dp;
  const S vel[3] = {qm[1] + 0.5 * dq[1], qm[2] + 0.5 * dq[2], qm[3] + 0.5 * dq[3]};
  const S T = qm[4] + 0.5 * dT;
  S iT = s_rcp(T);
  S rho = p * iT;
  S irho = T * s_rcp(p);
  S c2 = ph.gamma * T;
  S vv = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
  S e2 = s_min(S(1.0), s_max(S(ph.eps_min * ph.eps_min), vv * iT * ph.inv_gamma));
  S Ur2 = e2 * c2;
  S ie2 = s_rcp(e2);
  S iUr2 = ie2 * iT * ph.inv_gamma;
  S un = vel[0] * n[0] + vel[1] * n[1] + vel[2] * n[2];
  S dun = dvel[0] * n[0] + dvel[1] * n[1] + dvel[2] * n[2];
  S alpha = 0.5 * (1.0 - e2);
  S cpr = s_sqrt(alpha * alpha * un * un + Ur2);
  S unp = un * (1.0 - alpha);
  S lp = unp + cpr, lm = unp - cpr;
  S alp = s_abs(lp), alm = s_abs(lm), aun = s_abs(un);
  S a1 = (alp - alm) * (0.5 * s_rcp(cpr));
  S a0 = alp - a1 * lp;
  S rc2 = rho * c2;
  S zp = a0 * dp + a1 * (e2 * (un * dp + rc2 * dun));
  S zu = a0 * dun + a1 * (dp * irho + un * dun);
  S w0 = rho * dun;
  S w1 = (dp * irho + (1.0 - e2) * un * dun) * iUr2;
  S y0 = (a0 - aun) * w0 + a1 * (e2 * (un * w0 + rc2 * w1));
  S y1 = (a0 - aun) * w1 + a1 * (dun + un * w1);
  S irCp = irho / ph.Cp;
  S xT = -(1.0 - e2) * un * irCp * y0 + e2 * ph.gm1 * T * y1 + aun * dT;
  S xv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) xv[c] = zu * n[c] + aun * (dvel[c] - dun * n[c]);
  S yp = zp * ie2;
  S yT = (ie2 - 1.0) * irCp * zp + xT;
  S drho = (yp - rho * yT) * iT;
  S H = ph.Cp * T + 0.5 * vv;
  S d[5];
  d[0] = drho;
#pragma unroll
  for (int c = 0; c < 3; ++c) d[1 + c] = vel[c] * drho + rho * xv[c];
  d[4] = H * drho - yp + rho * (vel[0] * xv[0] + vel[1] * xv[1] + vel[2] * xv[2]) + rho * ph.Cp * yT;
  const double hdS = 0.5 * dS;
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = ((fm[v] + fp[v]) - d[v]) * hdS;
}

template <class S>
__host__ __device__ inline void roe3_flux(const S qm[5], const S qp[5], const double n[3], double dS, const Phys& ph,
                                          S out[5]) {
  S dq[5] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3], qp[4] - qm[4]};
  roe3_flux_jump(qm, qp, dq, qm[0] - ph.p_ref, qp[0] - ph.p_ref, n, dS, ph, out);
}

// Gamma (eq. preconditioning) and M = dq_c/dq_p at one point, row-major 5x5.
__host__ __device__ inline void gamma_and_M3(const double q[5], const Phys& ph, double G[25], double M[25]) {
  double p = q[0], T = q[4];
  double rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double H = ph.Cp * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double e2 = eps2_of3(q, ph);
  double Th = 1.0 / (e2 * ph.gamma * T) - rT / (rho * ph.Cp);
  double c0[5] = {1.0, q[1], q[2], q[3], H};
  for (int i = 0; i < 5; ++i) {
    G[i * 5 + 0] = Th * c0[i];
    M[i * 5 + 0] = rp * c0[i];
    G[i * 5 + 4] = M[i * 5 + 4] = rT * c0[i];
    for (int j = 1; j < 4; ++j) G[i * 5 + j] = M[i * 5 + j] = 0.0;
  }
  G[20] -= 1.0; M[20] -= 1.0;
  for (int c = 1; c < 4; ++c) {
    G[c * 5 + c] = M[c * 5 + c] = rho;
    G[20 + c] = M[20 + c] = rho * q[c];
  }
  G[24] += rho * ph.Cp;
  M[24] += rho * ph.Cp;
}

// Ghost state of a boundary face: slip wall (p, v - 2 (v.n) n, T) or far field
// (the free stream ph.qinf[0..4] = (p, u, v, w, T)).  n is the unit outward normal.
template <class S>
__host__ __device__ inline void ghost_state3(int bc, const S qm[5], const double n[3], const Phys& ph, S qg[5]) {
  if (bc == 4) {
    for (int v = 0; v < 5; ++v) qg[v] = S(ph.qinf[v]);
    return;
  }
  qg[0] = qm[0];
  qg[4] = qm[4];
  if (bc == 3) {   // no-slip adiabatic wall: velocity reversed
#pragma unroll
    for (int c = 0; c < 3; ++c) qg[1 + c] = -qm[1 + c];
    return;
  }
  const S un = qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) qg[1 + c] = qm[1 + c] - 2.0 * un * n[c];
}

// Viscous fluxes in 3D (Section 2.1) from the velocity (u0, u1, u2) and the
// gradients g[c*4 + k] = d(u, v, w, T)_k / dx_c: the stress tau_ij =
// mu (du_i/dx_j + du_j/dx_i) - (2/3) mu div(u) delta_ij and the heat flux
// kT dT/dx_c.  fv[c*4 + r] is the flux in direction c of row r + 1 (x-, y-,
// z-momentum, energy: u_i tau_ic + kT dT/dx_c); the mass row is zero.
template <class S>
__host__ __device__ inline void viscous_flux3(const S uvw[3], const S g[12], const Phys& ph, S fv[12]) {
  const S div3 = (g[0] + g[5] + g[10]) * (2.0 / 3.0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    S tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i] = ph.mu * (g[c * 4 + i] + g[i * 4 + c]);
    tau[c] = tau[c] - ph.mu * div3;
#pragma unroll
    for (int i = 0; i < 3; ++i) fv[c * 4 + i] = tau[i];
    fv[c * 4 + 3] = uvw[0] * tau[0] + uvw[1] * tau[1] + uvw[2] * tau[2] + ph.kT * g[c * 4 + 3];
  }
}

}  // namespace pmg
