// physics.cuh -- pointwise physics of the preconditioned Euler equations
// (Sections 2.1-2.3): fluxes, the preconditioning matrix, and the
// Weiss-Smith/Turkel preconditioned Roe flux in a closed form.
//
// All functions are templates over the scalar type S so that the same code
// gives values (S = double) and exact forward-mode derivatives (S = Dual)
// for the element-block assembly.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace pmg {

struct Phys {
  double gamma;    // ratio of specific heats
  double gm1;      // gamma - 1
  double Cp;       // gamma / (gamma - 1) with R = 1
  double eps_min;  // kappa * Ma_inf when the cut-off is on, 0 otherwise
  double p_ref;    // device states hold p - p_ref (gauge pressure)
  double inv_gamma;  // 1 / gamma
  double inv_gm1;    // 1 / (gamma - 1)
  double mu;         // constant dynamic viscosity (0: Euler)
  double kT;         // heat conductivity mu Cp / Pr
  double nw[5];      // weights 1 / res_scale of the equations in the residual norm
  double qinf[5];    // free stream of far-field faces: (p absolute, u, v, T) in 2D,
                     // (p absolute, u, v, w, T) in 3D
  double wait_ns;    // bound of the bulk-copy waits (< 0: give up at once)
};

// ---------------------------------------------------------------------------
// Forward-mode dual number with one derivative direction.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(double a) : v(a), d(0.0) {}
  __host__ __device__ Dual(double a, double b) : v(a), d(b) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  double r = 1.0 / b.v;
  double q = a.v * r;
  return Dual(q, (a.d - q * b.d) * r);
}
__host__ __device__ inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__host__ __device__ inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__host__ __device__ inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__host__ __device__ inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__host__ __device__ inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__host__ __device__ inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__host__ __device__ inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__host__ __device__ inline Dual operator/(double a, Dual b) {
  double r = 1.0 / b.v;
  double q = a * r;
  return Dual(q, -q * b.d * r);
}
__host__ __device__ inline double val(double a) { return a; }
__host__ __device__ inline double val(Dual a) { return a.v; }
__host__ __device__ inline double s_sqrt(double a) { return sqrt(a); }
__host__ __device__ inline Dual s_sqrt(Dual a) {
  double s = sqrt(a.v);
  return Dual(s, a.d * 0.5 / s);
}
__host__ __device__ inline double s_abs(double a) { return fabs(a); }
__host__ __device__ inline Dual s_abs(Dual a) { return a.v < 0.0 ? -a : a; }
// Reciprocal.  On the device, division costs about ten FP64 FMAs on GB300;
// here the hardware approximation (PTX rcp.approx.ftz.f64, about 20 correct
// bits) is refined by two Newton-Raphson steps y <- y + y (1 - x y), each
// doubling the number of correct bits, to full FP64 accuracy (within an ulp
// or two of the correctly rounded quotient; the parity tests bound the
// effect on the residual).  Arguments here are normal numbers (T, p, eps^2,
// c' > 0).  Dual numbers use plain division.
__host__ __device__ inline double s_rcp(double x) {
#ifdef __CUDA_ARCH__
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
#else
  return 1.0 / x;
#endif
}
__host__ __device__ inline Dual s_rcp(Dual x) { return 1.0 / x; }
template <class S> __host__ __device__ inline S s_min(S a, S b) { return val(a) <= val(b) ? a : b; }
template <class S> __host__ __device__ inline S s_max(S a, S b) { return val(a) >= val(b) ? a : b; }

// ---------------------------------------------------------------------------
// Inviscid flux through the unit direction (nx, ny):
// (rho u_n, rho u_n u + p nx, rho u_n v + p ny, rho u_n H), R = 1.
// ---------------------------------------------------------------------------
//
// q holds the absolute pressure; pm is the pressure used in the momentum
// flux.  With gauge storage pm = p - p_ref: the constant p_ref contributes
// p_ref times the discrete metric identity, which vanishes wherever the
// discretisation preserves a uniform flow (straight elements, or curved
// elements with P >= geometry order), and leaving it out keeps the rounding
// of p ~ 1/Ma^2 out of the momentum residual (and, through the velocity
// updates, out of the H-weighted energy residual).
template <class S>
__host__ __device__ inline void flux_n(const S q[4], const S& pm, double nx, double ny, const Phys& ph, S f[4]) {
  S rho = q[0] * s_rcp(q[3]);
  S H = ph.Cp * q[3] + 0.5 * (q[1] * q[1] + q[2] * q[2]);
  S mn = rho * (q[1] * nx + q[2] * ny);
  f[0] = mn;
  f[1] = mn * q[1] + pm * nx;
  f[2] = mn * q[2] + pm * ny;
  f[3] = mn * H;
}

// Cartesian fluxes f (x) and g (y) at one point (pm as in flux_n), with the
// density rho = p / T supplied by the caller.
template <class S>
__host__ __device__ inline void flux_xy_rho(const S q[4], const S& pm, const S& rho, const Phys& ph, S f[4],
                                            S g[4]) {
  S H = ph.Cp * q[3] + 0.5 * (q[1] * q[1] + q[2] * q[2]);
  S mx = rho * q[1], my = rho * q[2];
  f[0] = mx; f[1] = mx * q[1] + pm; f[2] = mx * q[2]; f[3] = mx * H;
  g[0] = my; g[1] = my * q[1]; g[2] = my * q[2] + pm; g[3] = my * H;
}

template <class S>
__host__ __device__ inline void flux_xy(const S q[4], const S& pm, const Phys& ph, S f[4], S g[4]) {
  flux_xy_rho(q, pm, q[0] * s_rcp(q[3]), ph, f, g);
}

// Conservative variables (rho, rho u, rho v, rho E).
template <class S>
__host__ __device__ inline void cons(const S q[4], const Phys& ph, S qc[4]) {
  S rho = q[0] / q[3];
  qc[0] = rho;
  qc[1] = rho * q[1];
  qc[2] = rho * q[2];
  qc[3] = rho * (q[3] * ph.inv_gm1 + 0.5 * (q[1] * q[1] + q[2] * q[2]));
}

// eps^2 with eps = min(1, max(eps_min, Ma)) (eq. eps_nonmove; eps_min = 0
// when the cut-off is off).
template <class S>
__host__ __device__ inline S eps2_of(const S q[4], const Phys& ph) {
  S ma2 = (q[1] * q[1] + q[2] * q[2]) / (ph.gamma * q[3]);
  S e2 = s_max(S(ph.eps_min * ph.eps_min), ma2);
  return s_min(S(1.0), e2);
}

// ---------------------------------------------------------------------------
// Preconditioned Roe flux (eq. invis_com) through unit normal (nx, ny) times
// the face area dS, with every matrix at the arithmetic mean of the primitive
// states.
//
// Closed form used here.  With K = M^-1 Gamma (identity except K_pp = 1/eps^2
// and K_Tp = (1/eps^2 - 1)/(rho Cp)), Gamma = M K and
// Gamma^-1 A_n = K^-1 (M^-1 A_n).  In rotated primitive variables
// (p, u_n, u_t, T) the matrix K^-1 M^-1 A_n is block lower triangular: a 2x2
// acoustic block B on (p, u_n) with eigenvalues u_n' +- c', u_t decoupled
// with eigenvalue u_n, and the T row coupled to (p, u_n) through
// r = (-(1-eps^2) u_n/(rho Cp), eps^2 (gamma-1) T) with eigenvalue u_n.  So
// |B| = a0 I + a1 B (linear interpolation of |lambda| on the two acoustic
// eigenvalues), and the T row of |.| is r (|B| - |u_n|)(B - u_n)^-1 on
// (p, u_n) plus |u_n| on T.  The dissipation is then M K |.| dq_p.
// ---------------------------------------------------------------------------
template <class S>
__host__ __device__ inline void roe_flux_jump(const S qm[4], const S qp[4], const S dq[4], const S& pmm,
                                              const S& pmp, double nx, double ny, double dS, const Phys& ph,
                                              S out[4]) {
  S fm[4], fp[4];
  flux_n(qm, pmm, nx, ny, ph, fm);
  flux_n(qp, pmp, nx, ny, ph, fp);
  // averaged state, formed from the jump: (q^- + q^+)/2 = q^- + dq/2
  S dp = dq[0], du = dq[1], dv = dq[2], dT = dq[3];
  S p = qm[0] + 0.5 * dp;
  S u = qm[1] + 0.5 * du;
  S v = qm[2] + 0.5 * dv;
  S T = qm[3] + 0.5 * dT;
  // divisions are ~10 FP64 FMA each on GB300: form each reciprocal once
  S iT = s_rcp(T);
  S rho = p * iT;
  S irho = T * s_rcp(p);
  S c2 = ph.gamma * T;
  S vv = u * u + v * v;
  S e2 = s_min(S(1.0), s_max(S(ph.eps_min * ph.eps_min), vv * iT * ph.inv_gamma));
  S Ur2 = e2 * c2;
  S ie2 = s_rcp(e2);
  S iUr2 = ie2 * iT * ph.inv_gamma;
  S un = u * nx + v * ny;
  S dun = du * nx + dv * ny;
  S dut = dv * nx - du * ny;
  S alpha = 0.5 * (1.0 - e2);
  S cpr = s_sqrt(alpha * alpha * un * un + Ur2);
  S unp = un * (1.0 - alpha);
  S lp = unp + cpr, lm = unp - cpr;
  S alp = s_abs(lp), alm = s_abs(lm), aun = s_abs(un);
  S a1 = (alp - alm) * (0.5 * s_rcp(cpr));
  S a0 = alp - a1 * lp;
  S rc2 = rho * c2;
  // |B| (dp, dun)
  S zp = a0 * dp + a1 * (e2 * (un * dp + rc2 * dun));
  S zu = a0 * dun + a1 * (dp * irho + un * dun);
  // w = (B - u_n)^-1 (dp, dun)
  S w0 = rho * dun;
  S w1 = (dp * irho + (1.0 - e2) * un * dun) * iUr2;
  // (|B| - |u_n|) w
  S y0 = (a0 - aun) * w0 + a1 * (e2 * (un * w0 + rc2 * w1));
  S y1 = (a0 - aun) * w1 + a1 * (dun + un * w1);   // w0 / rho = dun
  S irCp = irho / ph.Cp;
  S xT = -(1.0 - e2) * un * irCp * y0 + e2 * ph.gm1 * T * y1 + aun * dT;
  S xt = aun * dut;
  S xu = zu * nx - xt * ny;
  S xv = zu * ny + xt * nx;
  // K then M
  S yp = zp * ie2;
  S yT = (ie2 - 1.0) * irCp * zp + xT;
  S drho = (yp - rho * yT) * iT;
  S H = ph.Cp * T + 0.5 * vv;
  S d0 = drho;
  S d1 = u * drho + rho * xu;
  S d2 = v * drho + rho * xv;
  S d3 = H * drho - yp + rho * (u * xu + v * xv) + rho * ph.Cp * yT;
  const double hdS = 0.5 * dS;
  out[0] = ((fm[0] + fp[0]) - d0) * hdS;
  out[1] = ((fm[1] + fp[1]) - d1) * hdS;
  out[2] = ((fm[2] + fp[2]) - d2) * hdS;
  out[3] = ((fm[3] + fp[3]) - d3) * hdS;
}

// Same flux with the jump q_p^+ - q_p^- formed from the two traces.
template <class S>
__host__ __device__ inline void roe_flux(const S qm[4], const S qp[4], double nx, double ny, double dS,
                                         const Phys& ph, S out[4]) {
  S dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  roe_flux_jump(qm, qp, dq, qm[0] - ph.p_ref, qp[0] - ph.p_ref, nx, ny, dS, ph, out);
}

// Gamma (eq. preconditioning, 2D rows) and M = dq_c/dq_p at one point,
// row-major 4x4.
__host__ __device__ inline void gamma_and_M(const double q[4], const Phys& ph, double G[16], double M[16]) {
  double p = q[0], u = q[1], v = q[2], T = q[3];
  double rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double H = ph.Cp * T + 0.5 * (u * u + v * v);
  double e2 = eps2_of(q, ph);
  double Th = 1.0 / (e2 * ph.gamma * T) - rT / (rho * ph.Cp);
  double c0[4] = {1.0, u, v, H};
  for (int i = 0; i < 4; ++i) {
    G[i * 4 + 0] = Th * c0[i];
    M[i * 4 + 0] = rp * c0[i];
    G[i * 4 + 3] = rT * c0[i];
    M[i * 4 + 3] = rT * c0[i];
    G[i * 4 + 1] = G[i * 4 + 2] = M[i * 4 + 1] = M[i * 4 + 2] = 0.0;
  }
  G[12] -= 1.0; M[12] -= 1.0;
  G[5] = M[5] = rho;
  G[10] = M[10] = rho;
  G[13] = M[13] = rho * u;
  G[14] = M[14] = rho * v;
  G[15] += rho * ph.Cp;
  M[15] += rho * ph.Cp;
}

// Viscous fluxes (Section 2.1, constant mu) in x and y from the velocity and
// the gradients g = (du/dx, dv/dx, dT/dx, du/dy, dv/dy, dT/dy):
// tau_ij = mu (du_i/dx_j + du_j/dx_i) - (2/3) mu div(u) delta_ij, and the
// energy flux u_i tau_ij - K_j with K_j = -kT dT/dx_j.  Mass rows are zero.
template <class S>
__host__ __device__ inline void viscous_flux(S u, S v, const S g[6], const Phys& ph, S fv[4], S gv[4]) {
  const S div3 = (g[0] + g[4]) * (2.0 / 3.0);
  const S txx = ph.mu * (2.0 * g[0] - div3);
  const S tyy = ph.mu * (2.0 * g[4] - div3);
  const S txy = ph.mu * (g[3] + g[1]);
  fv[0] = 0.0;
  fv[1] = txx;
  fv[2] = txy;
  fv[3] = u * txx + v * txy + ph.kT * g[2];
  gv[0] = 0.0;
  gv[1] = txy;
  gv[2] = tyy;
  gv[3] = u * txy + v * tyy + ph.kT * g[5];
}

// Ghost state of a boundary face (the paper states no boundary treatment;
// reading: a ghost state enters the same common fluxes).  q holds absolute
// pressure; (nx, ny) is the unit outward normal.  bc 2: slip wall
// (p, u - 2 u_n n, T); 3: no-slip adiabatic wall (p, -u, -v, T); 4: far
// field (the free stream).
template <class S>
__host__ __device__ inline void ghost_state(int bc, const S qm[4], double nx, double ny, const Phys& ph, S qg[4]) {
  if (bc == 4) {
    for (int v = 0; v < 4; ++v) qg[v] = S(ph.qinf[v]);
    return;
  }
  qg[0] = qm[0];
  qg[3] = qm[3];
  if (bc == 3) {
    qg[1] = -qm[1];
    qg[2] = -qm[2];
  } else {
    const S un = qm[1] * nx + qm[2] * ny;
    qg[1] = qm[1] - 2.0 * un * nx;
    qg[2] = qm[2] - 2.0 * un * ny;
  }
}

}  // namespace pmg
