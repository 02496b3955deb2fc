// physics_dw.cuh -- the preconditioned Roe flux of physics.cuh (eq. invis_com,
// same closed form, same order of operations) in double-word arithmetic
// (dword.cuh), for the residual kernels.  GB300's FP64 rate (2 lanes per
// clock per SM) bounds the face-flux and sweep kernels; the same flux on the
// FP32 pipes runs several times faster at ~2^-46 relative rounding.
//
// The jumps dq arrive already formed in binary64 relative to a common
// reference (see line_trace in k_residual.cu): their double-word copies keep
// the low-Mach cancellation p+ - p- out of this arithmetic entirely.
#pragma once
#include "dword.cuh"
#include "physics.cuh"

namespace pmg {

// Double-word copies of the gas constants (filled on the host).
struct PhysW {
  dw gamma, Cp, gm1, inv_gamma, inv_Cp, eps_min2;
  dw p_ref;     // gauge reference pressure of the device states
  dw inv_gm1;   // 1 / (gamma - 1)
  double wait_ns;   // bound of the bulk-copy waits (< 0: give up at once)
};

// Double-word copies of a level's 1D operators (see OpTab).
struct OpTabW {
  dw D[6][6];
  dw lm[6], lp[6], gL[6], gR[6];
};

inline PhysW make_physw(const Phys& ph) {
  PhysW k;
  k.gamma = dw_const(ph.gamma);
  k.Cp = dw_const(ph.Cp);
  k.gm1 = dw_const(ph.gm1);
  k.inv_gamma = dw_const(ph.inv_gamma);
  k.inv_Cp = dw_const(1.0 / ph.Cp);
  k.eps_min2 = dw_const(ph.eps_min * ph.eps_min);
  k.p_ref = dw_const(ph.p_ref);
  k.inv_gm1 = dw_const(ph.inv_gm1);
  k.wait_ns = ph.wait_ns;
  return k;
}

#ifdef __CUDACC__
__device__ __forceinline__ dw half(dw x) { return scale2(x, 0.5f); }
__device__ __forceinline__ dw one_minus(dw x) { return dw{1.0f, 0.0f} - x; }

// Convective part of flux_n of physics.cuh: (rho u_n, rho u_n u, rho u_n v,
// rho u_n H); the pressure term pm n of the momentum rows is left to the
// caller.
__device__ __forceinline__ void flux_n_dw(const dw q[4], dw nx, dw ny, const PhysW& k, dw f[4]) {
  const dw rho = q[0] * rcp(q[3]);
  const dw H = k.Cp * q[3] + half(q[1] * q[1] + q[2] * q[2]);
  const dw mn = rho * (q[1] * nx + q[2] * ny);
  f[0] = mn;
  f[1] = mn * q[1];
  f[2] = mn * q[2];
  f[3] = mn * H;
}

// roe_flux_jump of physics.cuh in double-word, without the pressure part
// (pm^- + pm^+)/2 n dS of the central momentum flux: qm, qp hold absolute
// pressure, dq = qp - qm (formed by the caller), (nx, ny) is the unit normal
// and dS the face area.  The pressure part is the one large term of the
// momentum rows (p ~ 1/(gamma Ma^2) when the absolute pressure is stored);
// the caller adds it in binary64.
__device__ __forceinline__ void roe_flux_jump_dw(const dw qm[4], const dw qp[4], const dw dq[4], dw nx, dw ny,
                                                 dw dS, const PhysW& k, dw out[4]) {
  dw fm[4], fp[4];
  flux_n_dw(qm, nx, ny, k, fm);
  flux_n_dw(qp, nx, ny, k, fp);
  const dw dp = dq[0], du = dq[1], dv = dq[2], dT = dq[3];
  const dw p = qm[0] + half(dp);
  const dw u = qm[1] + half(du);
  const dw v = qm[2] + half(dv);
  const dw T = qm[3] + half(dT);
  const dw iT = rcp(T);
  const dw rho = p * iT;
  const dw irho = T * rcp(p);
  const dw c2 = k.gamma * T;
  const dw vv = u * u + v * v;
  const dw e2 = min_dw(dw{1.0f, 0.0f}, max_dw(k.eps_min2, vv * iT * k.inv_gamma));
  const dw Ur2 = e2 * c2;
  const dw ie2 = rcp(e2);
  const dw iUr2 = ie2 * iT * k.inv_gamma;
  const dw un = u * nx + v * ny;
  const dw dun = du * nx + dv * ny;
  const dw dut = dv * nx - du * ny;
  const dw ome2 = one_minus(e2);
  const dw alpha = half(ome2);
  const dw aun2 = alpha * un;
  const dw cpr = sqrt_dw(aun2 * aun2 + Ur2);
  const dw unp = un - aun2;
  const dw lp = unp + cpr, lm = unp - cpr;
  const dw alp = abs_dw(lp), alm = abs_dw(lm), aun = abs_dw(un);
  const dw a1 = (alp - alm) * half(rcp(cpr));
  const dw a0 = alp - a1 * lp;
  const dw rc2 = rho * c2;
  const dw dpr = dp * irho;
  // |B| (dp, dun)
  const dw zp = a0 * dp + a1 * (e2 * (un * dp + rc2 * dun));
  const dw zu = a0 * dun + a1 * (dpr + un * dun);
  // w = (B - u_n)^-1 (dp, dun)
  const dw w0 = rho * dun;
  const dw w1 = (dpr + ome2 * un * dun) * iUr2;
  // (|B| - |u_n|) w
  const dw a0u = a0 - aun;
  const dw y0 = a0u * w0 + a1 * (e2 * (un * w0 + rc2 * w1));
  const dw y1 = a0u * w1 + a1 * (dun + un * w1);
  const dw irCp = irho * k.inv_Cp;
  const dw xT = aun * dT + e2 * k.gm1 * T * y1 - ome2 * un * irCp * y0;
  const dw xt = aun * dut;
  const dw xu = zu * nx - xt * ny;
  const dw xv = zu * ny + xt * nx;
  // K then M
  const dw yp = zp * ie2;
  const dw yT = (ie2 - dw{1.0f, 0.0f}) * irCp * zp + xT;
  const dw drho = (yp - rho * yT) * iT;
  const dw H = k.Cp * T + half(vv);
  const dw d1 = u * drho + rho * xu;
  const dw d2 = v * drho + rho * xv;
  const dw d3 = H * drho - yp + rho * (u * xu + v * xv) + rho * k.Cp * yT;
  const dw hdS = half(dS);
  out[0] = ((fm[0] + fp[0]) - drho) * hdS;
  out[1] = ((fm[1] + fp[1]) - d1) * hdS;
  out[2] = ((fm[2] + fp[2]) - d2) * hdS;
  out[3] = ((fm[3] + fp[3]) - d3) * hdS;
}

// Common Roe flux of one face point from binary64 traces; DWF selects the
// double-word evaluation (above; the central pressure term in binary64)
// over the binary64 one.
template <bool DWF>
__device__ __forceinline__ void face_roe(const double qm[4], const double qp[4], const double dq[4], double pgm,
                                         double pgp, double nx, double ny, double dS, const Phys& ph,
                                         const PhysW& phw, double out[4]) {
  if (DWF) {
    dw Qm[4], Qp[4], DQ[4], o[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      Qm[v] = dw_from_double(qm[v]);
      Qp[v] = dw_from_double(qp[v]);
      DQ[v] = dw_from_double(dq[v]);
    }
    roe_flux_jump_dw(Qm, Qp, DQ, dw_from_double(nx), dw_from_double(ny), dw_from_double(dS), phw, o);
    const double pc = (pgm + pgp) * (0.5 * dS);
    out[0] = dw_to_double(o[0]);
    out[1] = fma(pc, nx, dw_to_double(o[1]));
    out[2] = fma(pc, ny, dw_to_double(o[2]));
    out[3] = dw_to_double(o[3]);
  } else {
    roe_flux_jump(qm, qp, dq, pgm, pgp, nx, ny, dS, ph, out);
  }
}
// The double-word face flux left in double-word, the central pressure term
// included: for gauge storage, where the momentum-flux pressures pgm, pgp
// are the small p - p_ref.
__device__ __forceinline__ void face_roe_dw(const double qm[4], const double qp[4], const double dq[4], double pgm,
                                            double pgp, double nx, double ny, double dS, const PhysW& phw,
                                            dw out[4]) {
  dw Qm[4], Qp[4], DQ[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    Qm[v] = dw_from_double(qm[v]);
    Qp[v] = dw_from_double(qp[v]);
    DQ[v] = dw_from_double(dq[v]);
  }
  const dw NX = dw_from_double(nx), NY = dw_from_double(ny), DS = dw_from_double(dS);
  roe_flux_jump_dw(Qm, Qp, DQ, NX, NY, DS, phw, out);
  const dw pc = half((dw_from_double(pgm) + dw_from_double(pgp)) * DS);
  out[1] = out[1] + pc * NX;
  out[2] = out[2] + pc * NY;
}
#endif  // __CUDACC__

}  // namespace pmg
