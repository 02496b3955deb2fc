// pmg_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of the implicit P-multigrid flux
// reconstruction solver of Wang & Yu (arXiv 1908.03972) for the 2D Euler and
// (constant mu, Section 2.1) Navier-Stokes equations with Weiss-Smith/Turkel
// local preconditioning.  Viscous terms follow Section 2.3: q_com of eq.
// com_q, common gradient of eq. com_grad_q with BR2 liftings.  The paper does
// not state the BR2 penalty; eta_f = 4 (the faces of a quadrilateral) is the
// reading taken, for hexahedra too, and its value is parity unpinned (every
// pin holds for any eta_f > 0).
// Boundary faces (slip wall, no-slip adiabatic wall, far field) use ghost
// states through the same common fluxes; the paper states none (reading).  It exists only to
// check the CUDA library: tests, the smoke check and the CPU-baseline leg of
// the benchmark may load it; the product path never does.  It shares no code,
// header, table or constant generator with the CUDA library.
//
// Every function cites the part of the paper it follows.  Where the paper is
// silent the reading taken is stated next to the code.  The residual is a
// template over the scalar type so that the block Jacobians can be taken by
// complex-step differentiation (exact to rounding, neighbours frozen).
//
// Layout conventions (shared with the library only through the C interface):
//   solution point (i, j) of a degree-P element has index j*(P+1)+i, i along xi;
//   a state array is variable-major: q[(v*E + e)*N + pt], v in (p, u, v, T);
//   an element block row/column index is v*N + pt;
//   faces: 0 eta=-1, 1 xi=+1, 2 eta=+1, 3 xi=-1; face points are ordered by the
//   tangential reference coordinate increasing.
//   nbr[(e*4+f)*3 + {0,1,2}] = (neighbour element, neighbour face, reversed?);
//   a boundary face has neighbour element -1 and the boundary type in the
//   second slot: 2 slip wall, 3 no-slip adiabatic wall, 4 far field.
//   Element geometry: (Ng+1)^2 Lagrange nodes at equispaced reference
//   positions, index b*(Ng+1)+a, a along xi; nodes[(e*(Ng+1)^2 + node)*2 + {x,y}].
#include <complex>
#include <vector>
#include <cmath>
#include <cstring>
#include <cstdio>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

// ---------------------------------------------------------------------------
// Scalar helpers that keep the residual analytic for the complex step.
// ---------------------------------------------------------------------------
static inline double re(double x) { return x; }
static inline double re(const cplx& x) { return x.real(); }
template <class S> static inline S cs_abs(const S& x) { return re(x) < 0 ? -x : x; }
template <class S> static inline S cs_min(const S& a, const S& b) { return re(a) <= re(b) ? a : b; }
template <class S> static inline S cs_max(const S& a, const S& b) { return re(a) >= re(b) ? a : b; }
static inline double cs_sqrt(double x) { return std::sqrt(x); }
static inline cplx cs_sqrt(const cplx& x) { return std::sqrt(x); }

// ---------------------------------------------------------------------------
// 1D reference element: Gauss-Legendre points, Lagrange basis, the DG
// (Radau) correction functions.  Section 2.3: tensor products of 1D
// correction polynomials on quadrilaterals.  Reading: solution points are the
// Gauss-Legendre points and g is the Radau polynomial that recovers nodal DG.
// ---------------------------------------------------------------------------
static void legendre(int n, double x, double* L, double* dL) {
  // Three-term recurrence (k+1) L_{k+1} = (2k+1) x L_k - k L_{k-1};
  // derivative from (1-x^2) L_n' = n (L_{n-1} - x L_n), with the endpoint value
  // L_n'(+-1) = (+-1)^{n-1} n(n+1)/2.
  double l0 = 1.0, l1 = x;
  if (n == 0) { *L = 1.0; *dL = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    l0 = l1; l1 = l2;
  }
  *L = l1;
  if (std::fabs(std::fabs(x) - 1.0) < 1e-15) {
    double s = (x > 0) ? 1.0 : ((n - 1) % 2 == 0 ? 1.0 : -1.0);
    *dL = s * n * (n + 1) / 2.0;
  } else {
    *dL = n * (l0 - x * l1) / (1.0 - x * x);
  }
}

struct Basis1D {
  int P;
  std::vector<double> x, w;        // P+1 Gauss-Legendre points, weights
  std::vector<double> D;           // D[i*(P+1)+k] = l_k'(x_i)
  std::vector<double> lm, lp;      // l_k(-1), l_k(+1)
  std::vector<double> gL, gR;      // g_L'(x_i), g_R'(x_i)
};

static double lagrange(const std::vector<double>& x, int k, double t) {
  double v = 1.0;
  for (size_t m = 0; m < x.size(); ++m)
    if ((int)m != k) v *= (t - x[m]) / (x[k] - x[m]);
  return v;
}

static double lagrange_deriv(const std::vector<double>& x, int k, double t) {
  // d/dt of prod_{m!=k} (t-x_m)/(x_k-x_m), by the product rule.
  double s = 0.0;
  for (size_t j = 0; j < x.size(); ++j) {
    if ((int)j == k) continue;
    double term = 1.0 / (x[k] - x[j]);
    for (size_t m = 0; m < x.size(); ++m)
      if ((int)m != k && m != j) term *= (t - x[m]) / (x[k] - x[m]);
    s += term;
  }
  return s;
}

static Basis1D make_basis(int P) {
  Basis1D b;
  b.P = P;
  int n = P + 1;
  b.x.resize(n); b.w.resize(n);
  for (int i = 0; i < n; ++i) {
    // Newton on L_n from the Chebyshev-like initial guess, ascending order.
    double t = -std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(n, t, &L, &dL);
      double dt = L / dL;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double L, dL;
    legendre(n, t, &L, &dL);
    b.x[i] = t;
    b.w[i] = 2.0 / ((1.0 - t * t) * dL * dL);
  }
  b.D.resize(n * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) b.D[i * n + k] = lagrange_deriv(b.x, k, b.x[i]);
  b.lm.resize(n); b.lp.resize(n);
  for (int k = 0; k < n; ++k) { b.lm[k] = lagrange(b.x, k, -1.0); b.lp[k] = lagrange(b.x, k, 1.0); }
  // g_L = (-1)^P/2 (L_P - L_{P+1}), g_R = 1/2 (L_P + L_{P+1}): degree P+1,
  // g_L(-1)=1, g_L(1)=0, g_R mirrored, both orthogonal to degree P-1.
  b.gL.resize(n); b.gR.resize(n);
  double sgn = (P % 2 == 0) ? 1.0 : -1.0;
  for (int i = 0; i < n; ++i) {
    double L0, dL0, L1, dL1;
    legendre(P, b.x[i], &L0, &dL0);
    legendre(P + 1, b.x[i], &L1, &dL1);
    b.gL[i] = 0.5 * sgn * (dL0 - dL1);
    b.gR[i] = 0.5 * (dL0 + dL1);
  }
  return b;
}

// Dense real Gaussian elimination with partial pivoting (used for the small
// mass-matrix solves and for the block LU of Section 2.4).
static bool lu_factor(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return true;
}

static void lu_solve(int n, const double* LU, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
    b[i] /= LU[i * n + i];
  }
}

// Restriction = L2 projection onto degree Pc in reference coordinates (the
// projection operator of Section 3), built from the mass matrix with the fine
// Gauss quadrature, which integrates degree Pc+Pf exactly.
static std::vector<double> make_restriction(const Basis1D& f, const Basis1D& c) {
  int nf = f.P + 1, nc = c.P + 1;
  std::vector<double> Mc(nc * nc, 0.0), B(nc * nf, 0.0);
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j)
      for (int q = 0; q < nf; ++q)
        Mc[i * nc + j] += f.w[q] * lagrange(c.x, i, f.x[q]) * lagrange(c.x, j, f.x[q]);
  for (int i = 0; i < nc; ++i)
    for (int q = 0; q < nf; ++q) B[i * nf + q] = f.w[q] * lagrange(c.x, i, f.x[q]);
  std::vector<int> piv(nc);
  lu_factor(nc, Mc.data(), piv.data());
  std::vector<double> R(nc * nf);
  std::vector<double> col(nc);
  for (int q = 0; q < nf; ++q) {
    for (int i = 0; i < nc; ++i) col[i] = B[i * nf + q];
    lu_solve(nc, Mc.data(), piv.data(), col.data());
    for (int i = 0; i < nc; ++i) R[i * nf + q] = col[i];
  }
  return R;
}

// Prolongation = evaluation of the coarse Lagrange polynomial at the fine points.
static std::vector<double> make_prolongation(const Basis1D& f, const Basis1D& c) {
  int nf = f.P + 1, nc = c.P + 1;
  std::vector<double> I(nf * nc);
  for (int i = 0; i < nf; ++i)
    for (int k = 0; k < nc; ++k) I[i * nc + k] = lagrange(c.x, k, f.x[i]);
  return I;
}

// ---------------------------------------------------------------------------
// Thermodynamics and preconditioning, Sections 2.1-2.2.  Nondimensional ideal
// gas with R = 1: rho = p/T, E = T/(gamma-1) + |v|^2/2, H = E + p/rho,
// c^2 = gamma T, Cp = gamma/(gamma-1).  Working variables q_p = (p, u, v, T).
// ---------------------------------------------------------------------------
struct Phys {
  double gamma, Ma_inf, kappa;
  int cutoff;  // 1: eps = min(1, max(kappa Ma_inf, Ma)); 0: eps = min(1, Ma)
  double mu = 0.0, Pr = 0.72;   // constant dynamic viscosity (0: Euler), Prandtl number
};

template <class S> static void cons_from_prim(const S q[4], const Phys& ph, S qc[4]) {
  S rho = q[0] / q[3];
  S E = q[3] / (ph.gamma - 1.0) + 0.5 * (q[1] * q[1] + q[2] * q[2]);
  qc[0] = rho; qc[1] = rho * q[1]; qc[2] = rho * q[2]; qc[3] = rho * E;
}

static void prim_from_cons(const double qc[4], const Phys& ph, double q[4]) {
  double rho = qc[0], u = qc[1] / rho, v = qc[2] / rho;
  double p = (ph.gamma - 1.0) * (qc[3] - 0.5 * rho * (u * u + v * v));
  q[0] = p; q[1] = u; q[2] = v; q[3] = p / rho;
}

// M = dq_c/dq_p written out (Section 2.2).
template <class S> static void M_matrix(const S q[4], const Phys& ph, S M[4][4]) {
  S p = q[0], u = q[1], v = q[2], T = q[3];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (u * u + v * v);
  M[0][0] = rp;           M[0][1] = 0.0;     M[0][2] = 0.0;     M[0][3] = rT;
  M[1][0] = rp * u;       M[1][1] = rho;     M[1][2] = 0.0;     M[1][3] = rT * u;
  M[2][0] = rp * v;       M[2][1] = 0.0;     M[2][2] = rho;     M[2][3] = rT * v;
  M[3][0] = rp * H - 1.0; M[3][1] = rho * u; M[3][2] = rho * v; M[3][3] = rT * H + rho * Cp;
}

// eps of eq. eps_nonmove; with the cut-off off, eps is the local Mach number
// (Section 4.1).  Reading: no lower floor.
template <class S> static S precond_eps(const S q[4], const Phys& ph) {
  S Ma = cs_sqrt((q[1] * q[1] + q[2] * q[2]) / (ph.gamma * q[3]));
  S e = ph.cutoff ? cs_max(S(ph.kappa * ph.Ma_inf), Ma) : Ma;
  return cs_min(S(1.0), e);
}

// Gamma of eq. preconditioning (2D rows), Theta of eq. theta, U_r = eps c.
template <class S> static void Gamma_matrix(const S q[4], const S& eps, const Phys& ph, S G[4][4]) {
  S p = q[0], u = q[1], v = q[2], T = q[3];
  S rho = p / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (u * u + v * v);
  S c2 = ph.gamma * T;
  S Ur2 = eps * eps * c2;
  S Th = 1.0 / Ur2 - rT / (rho * Cp);
  G[0][0] = Th;           G[0][1] = 0.0;     G[0][2] = 0.0;     G[0][3] = rT;
  G[1][0] = Th * u;       G[1][1] = rho;     G[1][2] = 0.0;     G[1][3] = rT * u;
  G[2][0] = Th * v;       G[2][1] = 0.0;     G[2][2] = rho;     G[2][3] = rT * v;
  G[3][0] = Th * H - 1.0; G[3][1] = rho * u; G[3][2] = rho * v; G[3][3] = rT * H + rho * Cp;
}

// Inviscid flux through a (possibly unnormalised) direction (nx, ny):
// (rho u_n, rho u_n u + p nx, rho u_n v + p ny, rho u_n H), Section 2.1.
template <class S> static void euler_flux_n(const S q[4], double nx, double ny, const Phys& ph, S f[4]) {
  S p = q[0], u = q[1], v = q[2], T = q[3];
  S rho = p / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (u * u + v * v);
  S un = u * nx + v * ny;
  f[0] = rho * un;
  f[1] = rho * un * u + p * nx;
  f[2] = rho * un * v + p * ny;
  f[3] = rho * un * H;
}

// A_n = d f_n / d q_p, differentiated by hand from euler_flux_n.
template <class S> static void flux_jacobian_n(const S q[4], double nx, double ny, const Phys& ph, S A[4][4]) {
  S p = q[0], u = q[1], v = q[2], T = q[3];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (u * u + v * v);
  S un = u * nx + v * ny;
  A[0][0] = rp * un;          A[0][1] = rho * nx;                A[0][2] = rho * ny;                A[0][3] = rT * un;
  A[1][0] = rp * un * u + nx; A[1][1] = rho * un + rho * u * nx; A[1][2] = rho * u * ny;            A[1][3] = rT * un * u;
  A[2][0] = rp * un * v + ny; A[2][1] = rho * v * nx;            A[2][2] = rho * un + rho * v * ny; A[2][3] = rT * un * v;
  A[3][0] = rp * un * H;      A[3][1] = rho * nx * H + rho * un * u;
  A[3][2] = rho * ny * H + rho * un * v;                         A[3][3] = rT * un * H + rho * un * Cp;
}

// Solve G X = A for the 4x4 X by elimination with partial pivoting on the real part.
template <class S> static void solve4(S G[4][4], S A[4][4], S X[4][4]) {
  S a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) { a[i][j] = G[i][j]; a[i][4 + j] = A[i][j]; }
  for (int k = 0; k < 4; ++k) {
    int p = k;
    for (int i = k + 1; i < 4; ++i)
      if (std::fabs(re(a[i][k])) > std::fabs(re(a[p][k]))) p = i;
    if (p != k) for (int j = 0; j < 8; ++j) std::swap(a[k][j], a[p][j]);
    for (int i = k + 1; i < 4; ++i) {
      S l = a[i][k] / a[k][k];
      for (int j = k; j < 8; ++j) a[i][j] -= l * a[k][j];
    }
  }
  for (int c = 0; c < 4; ++c)
    for (int i = 3; i >= 0; --i) {
      S s = a[i][4 + c];
      for (int j = i + 1; j < 4; ++j) s -= a[i][j] * X[j][c];
      X[i][c] = s / a[i][i];
    }
}

// Preconditioned Roe flux, eq. invis_com: the central average minus
// Gamma R|Lambda|R^-1 (q_p^+ - q_p^-)/2, with every matrix evaluated at the
// arithmetic mean of the two primitive states (reading of "averaged values";
// no entropy fix).  |Gamma^-1 A_n| is formed with Sylvester's formula from the
// three distinct eigenvalues u_n, u_n' +- c' of eq. eigenvalues_para, which
// needs no eigenvectors.  (Sx, Sy) is the area-scaled normal from - to +; the
// result is the flux through that area.
template <class S>
static void roe_flux(const S qm[4], const S qp[4], double Sx, double Sy, const Phys& ph, S out[4]) {
  double dS = std::sqrt(Sx * Sx + Sy * Sy);
  double nx = Sx / dS, ny = Sy / dS;
  S qa[4];
  for (int k = 0; k < 4; ++k) qa[k] = 0.5 * (qm[k] + qp[k]);
  S eps = precond_eps(qa, ph);
  S G[4][4], A[4][4], Mt[4][4];
  Gamma_matrix(qa, eps, ph, G);
  flux_jacobian_n(qa, nx, ny, ph, A);
  solve4(G, A, Mt);
  // eigenvalues, eq. eigenvalues_para
  S p = qa[0], T = qa[3];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S c = cs_sqrt(ph.gamma * T);
  S Ur = eps * c;
  S un = qa[1] * nx + qa[2] * ny;
  S beta = rp + rT / (rho * Cp);
  S alpha = 0.5 * (1.0 - beta * Ur * Ur);
  S cpr = cs_sqrt(alpha * alpha * un * un + Ur * Ur);
  S unp = un * (1.0 - alpha);
  S lam[3] = {un, unp + cpr, unp - cpr};
  S absM[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) absM[i][j] = 0.0;
  for (int k = 0; k < 3; ++k) {
    S Pk[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) Pk[i][j] = (i == j) ? S(1.0) : S(0.0);
    for (int jj = 0; jj < 3; ++jj) {
      if (jj == k) continue;
      S fac[4][4], tmp[4][4];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
          fac[i][j] = (Mt[i][j] - (i == j ? lam[jj] : S(0.0))) / (lam[k] - lam[jj]);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          S s = 0.0;
          for (int m = 0; m < 4; ++m) s += Pk[i][m] * fac[m][j];
          tmp[i][j] = s;
        }
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Pk[i][j] = tmp[i][j];
    }
    S al = cs_abs(lam[k]);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) absM[i][j] += al * Pk[i][j];
  }
  S dq[4], t1[4], diss[4];
  for (int k = 0; k < 4; ++k) dq[k] = qp[k] - qm[k];
  for (int i = 0; i < 4; ++i) {
    S s = 0.0;
    for (int j = 0; j < 4; ++j) s += absM[i][j] * dq[j];
    t1[i] = s;
  }
  for (int i = 0; i < 4; ++i) {
    S s = 0.0;
    for (int j = 0; j < 4; ++j) s += G[i][j] * t1[j];
    diss[i] = s;
  }
  S fm[4], fp[4];
  euler_flux_n(qm, nx, ny, ph, fm);
  euler_flux_n(qp, nx, ny, ph, fp);
  for (int k = 0; k < 4; ++k) out[k] = (0.5 * (fm[k] + fp[k]) - 0.5 * diss[k]) * dS;
}

// ---------------------------------------------------------------------------
// Geometry: Lagrange mapping of order Ng on equispaced reference nodes.
// Reading: every P-level evaluates the exact mapping at its own points.
// ---------------------------------------------------------------------------
struct LevelGeom {
  int P, N;
  Basis1D b;
  std::vector<double> met;   // per (e, pt): x_xi, x_eta, y_xi, y_eta, |J|
  std::vector<double> fS;    // per (e, face, k): outward area-scaled normal (Sx, Sy)
  std::vector<double> fJ;    // per (e, face, k): |J| of the element map at the face point
};

static void map_derivs(int Ng, const double* xn, double xi, double eta,
                       double* x_xi, double* x_eta, double* y_xi, double* y_eta) {
  std::vector<double> r(Ng + 1);
  for (int a = 0; a <= Ng; ++a) r[a] = -1.0 + 2.0 * a / (Ng > 0 ? Ng : 1);
  *x_xi = *x_eta = *y_xi = *y_eta = 0.0;
  for (int b = 0; b <= Ng; ++b)
    for (int a = 0; a <= Ng; ++a) {
      double la = lagrange(r, a, xi), lb = lagrange(r, b, eta);
      double da = lagrange_deriv(r, a, xi), db = lagrange_deriv(r, b, eta);
      const double* X = xn + (b * (Ng + 1) + a) * 2;
      *x_xi += da * lb * X[0]; *x_eta += la * db * X[0];
      *y_xi += da * lb * X[1]; *y_eta += la * db * X[1];
    }
}

// Point of the element map at (xi, eta).
static void map_point(int Ng, const double* xn, double xi, double eta, double* x, double* y) {
  std::vector<double> r(Ng + 1);
  for (int a = 0; a <= Ng; ++a) r[a] = -1.0 + 2.0 * a / (Ng > 0 ? Ng : 1);
  *x = *y = 0.0;
  for (int b = 0; b <= Ng; ++b)
    for (int a = 0; a <= Ng; ++a) {
      double phi = lagrange(r, a, xi) * lagrange(r, b, eta);
      *x += phi * xn[(b * (Ng + 1) + a) * 2];
      *y += phi * xn[(b * (Ng + 1) + a) * 2 + 1];
    }
}

// Element size of the CFL definition (Section 2.4): twice the minimum distance
// from the element's barycentre to its faces.  Reading: the barycentre is the
// area centroid (8-point Gauss quadrature of the mapped element); each face
// curve is sampled at 65 equispaced reference points and the distance is the
// smallest point-to-segment distance of that polyline.
static double element_dx(int Ng, const double* xn) {
  const Basis1D q8 = make_basis(7);
  double A = 0.0, cx = 0.0, cy = 0.0;
  for (int j = 0; j < 8; ++j)
    for (int i = 0; i < 8; ++i) {
      double a, b, c, d, x, y;
      map_derivs(Ng, xn, q8.x[i], q8.x[j], &a, &b, &c, &d);
      map_point(Ng, xn, q8.x[i], q8.x[j], &x, &y);
      double w = q8.w[i] * q8.w[j] * (a * d - b * c);
      A += w; cx += w * x; cy += w * y;
    }
  cx /= A; cy /= A;
  const int K = 64;
  double best = 1e300;
  for (int f = 0; f < 4; ++f) {
    double px = 0, py = 0;
    for (int k = 0; k <= K; ++k) {
      double t = -1.0 + 2.0 * k / K, xi, eta, x, y;
      if (f == 0) { xi = t; eta = -1.0; } else if (f == 1) { xi = 1.0; eta = t; }
      else if (f == 2) { xi = t; eta = 1.0; } else { xi = -1.0; eta = t; }
      map_point(Ng, xn, xi, eta, &x, &y);
      if (k > 0) {   // distance from (cx, cy) to the segment (px, py)-(x, y)
        double ex = x - px, ey = y - py, L2 = ex * ex + ey * ey;
        double s = L2 > 0 ? ((cx - px) * ex + (cy - py) * ey) / L2 : 0.0;
        s = std::min(1.0, std::max(0.0, s));
        double dx = px + s * ex - cx, dy = py + s * ey - cy;
        best = std::min(best, std::sqrt(dx * dx + dy * dy));
      }
      px = x; py = y;
    }
  }
  return 2.0 * best;
}

// ---------------------------------------------------------------------------
// Solver context
// ---------------------------------------------------------------------------
struct OrcConfig {
  int n_levels;
  int P[8];
  int n_smooth[8];
  double gamma, Ma_inf, kappa;
  int cutoff;
  int esdirk_stages;      // 4 = ESDIRK3 (the scheme implemented)
  double dtau_init, dtau_max, tol;
  int refresh_every, max_pseudo;
  double mu, Pr;
  double res_scale[4];    // reference scale of each equation in ||F|| (0: 1)
  double q_inf[4];        // free-stream primitive state (p, u, v, T) of far-field faces
  int cfl_mode;           // 1: dtau = CFL dtau_min (eq. CFL), SER on the CFL number
  double cfl_init, cfl_max;
  int refresh_always;     // 1: rebuild every refresh_every iterations throughout (Section 4.1)
};

struct Level {
  LevelGeom g;
  std::vector<double> q, qb, S, F;        // state, restricted state, forcing, residual
  std::vector<double> lu;                 // per element n*n LU factors
  std::vector<int> piv;
};

struct Oracle {
  OrcConfig cfg;
  Phys ph;
  int E, Ng;
  std::vector<double> nodes;
  std::vector<int> nbr;
  std::vector<Level> lev;
  std::vector<std::vector<double>> Rm, Pm;   // restriction / prolongation 1D, level l -> l+1
  std::vector<double> dx;                    // element size of eq. CFL (twice barycentre-to-face distance)
  // stage data (finest level)
  std::vector<double> src;                   // (q_c^n + dt sum a_ij R^j)/(omega dt)
  double omega_dt;
  double dtau;
  // ESDIRK3 tableau
  double A[6][6], b[6], c[6];
  int s;
};

static void build_level_geom(Oracle* o, int P, LevelGeom* g) {
  g->P = P; g->N = (P + 1) * (P + 1);
  g->b = make_basis(P);
  int n1 = P + 1, E = o->E, Ng = o->Ng, nn = (Ng + 1) * (Ng + 1);
  g->met.assign((size_t)E * g->N * 5, 0.0);
  g->fS.assign((size_t)E * 4 * n1 * 2, 0.0);
  g->fJ.assign((size_t)E * 4 * n1, 0.0);
  for (int e = 0; e < E; ++e) {
    const double* xn = &o->nodes[(size_t)e * nn * 2];
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        double a, bb, c, d;
        map_derivs(Ng, xn, g->b.x[i], g->b.x[j], &a, &bb, &c, &d);
        double* m = &g->met[((size_t)e * g->N + j * n1 + i) * 5];
        m[0] = a; m[1] = bb; m[2] = c; m[3] = d; m[4] = a * d - bb * c;
      }
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < n1; ++k) {
        double xi, eta;
        if (f == 0) { xi = g->b.x[k]; eta = -1.0; }
        else if (f == 1) { xi = 1.0; eta = g->b.x[k]; }
        else if (f == 2) { xi = g->b.x[k]; eta = 1.0; }
        else { xi = -1.0; eta = g->b.x[k]; }
        double x_xi, x_eta, y_xi, y_eta;
        map_derivs(Ng, xn, xi, eta, &x_xi, &x_eta, &y_xi, &y_eta);
        double Sx, Sy;
        if (f == 0) { Sx = y_xi; Sy = -x_xi; }          // -(grad eta)|J|
        else if (f == 1) { Sx = y_eta; Sy = -x_eta; }   // +(grad xi)|J|
        else if (f == 2) { Sx = -y_xi; Sy = x_xi; }     // +(grad eta)|J|
        else { Sx = -y_eta; Sy = x_eta; }               // -(grad xi)|J|
        double* s = &g->fS[(((size_t)e * 4 + f) * n1 + k) * 2];
        s[0] = Sx; s[1] = Sy;
        g->fJ[((size_t)e * 4 + f) * n1 + k] = x_xi * y_eta - x_eta * y_xi;
      }
  }
}

// Point index along the line normal to face f through face point k, at
// position m along the normal direction.
static inline int line_pt(int P, int f, int k, int m) {
  int n1 = P + 1;
  if (f == 0 || f == 2) return m * n1 + k;   // i = k, j = m
  return k * n1 + m;                          // j = k, i = m
}

// Trace of a state (one element, variable-major with stride N) at face point
// (f, k): extrapolation of the solution polynomial along the normal line.
template <class S>
static void trace_state(const Basis1D& b, const S* qe, int N, int f, int k, S out[4]) {
  int n1 = b.P + 1;
  const std::vector<double>& l = (f == 1 || f == 2) ? b.lp : b.lm;
  for (int v = 0; v < 4; ++v) {
    S s = 0.0;
    for (int m = 0; m < n1; ++m) s += l[m] * qe[v * N + line_pt(b.P, f, k, m)];
    out[v] = s;
  }
}

// Broken (uncorrected) gradient of one element's state at its solution
// points: reference derivatives by the Lagrange derivative matrix, then the
// chain rule with the exact metric terms.  g[(c*4 + v)*N + pt], c = x, y.
template <class S>
static void broken_gradient(const Level& L, int e, const S* qe, S* g) {
  const Basis1D& b = L.g.b;
  int n1 = b.P + 1, N = L.g.N;
  for (int v = 0; v < 4; ++v)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        S qx = 0.0, qy = 0.0;
        for (int m = 0; m < n1; ++m) {
          qx += b.D[i * n1 + m] * qe[v * N + j * n1 + m];
          qy += b.D[j * n1 + m] * qe[v * N + m * n1 + i];
        }
        const double* mt = &L.g.met[((size_t)e * N + j * n1 + i) * 5];
        int pt = j * n1 + i;
        g[(0 * 4 + v) * N + pt] = (mt[3] * qx - mt[2] * qy) / mt[4];
        g[(1 * 4 + v) * N + pt] = (-mt[1] * qx + mt[0] * qy) / mt[4];
      }
}

// Frozen neighbour data at every element face point, NT values each: the
// neighbour's state trace (4), its broken-gradient trace (8, x then y per
// variable) and its |J| at that face point.
static const int NT = 13;

static void neighbour_traces(const Oracle* o, const Level& L, const double* q, std::vector<double>& tr) {
  int P = L.g.P, n1 = P + 1, N = L.g.N, E = o->E;
  tr.assign((size_t)E * 4 * n1 * NT, 0.0);
  std::vector<double> qe(4 * N), g(8 * N);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f) {
      int en = o->nbr[(e * 4 + f) * 3 + 0], fn = o->nbr[(e * 4 + f) * 3 + 1];
      int rev = o->nbr[(e * 4 + f) * 3 + 2];
      if (en < 0) continue;   // boundary face: the ghost state follows the own trace
      for (int v = 0; v < 4; ++v)
        for (int p = 0; p < N; ++p) qe[v * N + p] = q[((size_t)v * E + en) * N + p];
      if (o->ph.mu > 0.0) broken_gradient<double>(L, en, qe.data(), g.data());
      for (int k = 0; k < n1; ++k) {
        int kn = rev ? P - k : k;
        double* t = &tr[(((size_t)e * 4 + f) * n1 + k) * NT];
        trace_state(L.g.b, qe.data(), N, fn, kn, t);
        if (o->ph.mu > 0.0) {
          trace_state(L.g.b, g.data(), N, fn, kn, t + 4);
          trace_state(L.g.b, g.data() + 4 * N, N, fn, kn, t + 8);
        }
        t[12] = L.g.fJ[((size_t)en * 4 + fn) * n1 + kn];
      }
    }
}

// Viscous fluxes (Section 2.1) in x and y from the state and the gradients
// d = (dp/dx, du/dx, dv/dx, dT/dx, dp/dy, du/dy, dv/dy, dT/dy): stress
// tau_ij = mu (du_i/dx_j + du_j/dx_i - 2/3 div u delta_ij), heat flux
// K_j = -(mu Cp / Pr) dT/dx_j, energy flux u_i tau_ij - K_j.
template <class S>
static void viscous_flux(const S q[4], const S d[8], const Phys& ph, S fv[4], S gv[4]) {
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S ux = d[1], vx = d[2], Tx = d[3], uy = d[5], vy = d[6], Ty = d[7];
  S dv = ux + vy;
  S txx = ph.mu * (2.0 * ux - (2.0 / 3.0) * dv);
  S tyy = ph.mu * (2.0 * vy - (2.0 / 3.0) * dv);
  S txy = ph.mu * (uy + vx);
  double k = ph.mu * Cp / ph.Pr;
  fv[0] = 0.0; fv[1] = txx; fv[2] = txy; fv[3] = q[1] * txx + q[2] * txy + k * Tx;
  gv[0] = 0.0; gv[1] = txy; gv[2] = tyy; gv[3] = q[1] * txy + q[2] * tyy + k * Ty;
}

// Boundary faces (the paper states no boundary treatment; reading: a ghost
// state enters the same common fluxes).  From the own trace q^- and the unit
// outward normal: slip wall (p, u - 2 u_n n, T); no-slip adiabatic wall
// (p, -u, T); far field the free stream.  For the viscous terms the ghost
// side mirrors the element (its broken-gradient trace and |J| are the own
// ones), which makes eq. com_grad_q the standard one-sided BR2 gradient
// grad q^- + eta_f g'(1) (q_com - q^-) S/|J|; walls carry no viscous energy
// flux (u_com = 0 on a no-slip wall and the wall is adiabatic).
template <class S>
static void ghost_state(int bc, const S qm[4], double nx, double ny, const double qinf[4], S qg[4]) {
  if (bc == 4) {
    for (int v = 0; v < 4; ++v) qg[v] = qinf[v];
    return;
  }
  qg[0] = qm[0];
  qg[3] = qm[3];
  if (bc == 3) {
    qg[1] = -qm[1];
    qg[2] = -qm[2];
  } else {
    S un = qm[1] * nx + qm[2] * ny;
    qg[1] = qm[1] - 2.0 * un * nx;
    qg[2] = qm[2] - 2.0 * un * ny;
  }
}

// FR/CPR residual R = -div f of one element (Section 2.3, eq. eqn:FR_diff):
// contravariant fluxes at solution points, Lagrange derivative, and the DG
// correction of the jumps between the common and the local (extrapolated flux
// polynomial) normal fluxes at the flux points.  Neighbour data are frozen.
//
// With mu > 0 the flux is f_inv - f_vis (Section 2.1).  The viscous flux at a
// solution point takes the corrected gradient: the reference derivatives of
// the state plus the DG correction of the jumps q_com - q^- (eq. com_q) at the
// flux points of the same line, then the chain rule.  At a flux point it takes
// q_com and the common gradient of eq. com_grad_q, with the BR2 liftings
// r^(+-) = eta_f g'(face) (q_com - q^(+-)) S^(+-) / |J|^(+-): the correction
// of that face alone, evaluated at the face point (g'_R(1) = (P+1)^2 / 2 for
// the DG correction; S the outward face normal scaled by the face metric).
template <class S>
static void element_residual(const Oracle* o, const Level& L, int e, const S* qe,
                             const double* ntr, S* Re) {
  const Basis1D& b = L.g.b;
  int P = b.P, n1 = P + 1, N = L.g.N;
  const Phys& ph = o->ph;
  const bool visc = ph.mu > 0.0;
  const double eta_f = 4.0, gface = 0.5 * n1 * n1;
  std::vector<S> Ft(4 * N), Gt(4 * N);
  // Viscous preliminaries: traces, common states, corrected gradients.
  std::vector<S> qm_all(4 * n1 * 4), qc_all(4 * n1 * 4), gb(8 * N), gc(8 * N);
  std::vector<S> qp_all(4 * n1 * 4);
  for (int f = 0; f < 4; ++f) {
    const int en = o->nbr[(e * 4 + f) * 3 + 0], bc = o->nbr[(e * 4 + f) * 3 + 1];
    for (int k = 0; k < n1; ++k) {
      S* qm = &qm_all[(f * n1 + k) * 4];
      S* qp = &qp_all[(f * n1 + k) * 4];
      trace_state(b, qe, N, f, k, qm);
      const double* t = &ntr[(((size_t)e * 4 + f) * n1 + k) * NT];
      if (en < 0) {
        const double* Sv = &L.g.fS[(((size_t)e * 4 + f) * n1 + k) * 2];
        const double dS = std::sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1]);
        ghost_state(bc, qm, Sv[0] / dS, Sv[1] / dS, o->cfg.q_inf, qp);
      } else {
        for (int v = 0; v < 4; ++v) qp[v] = t[v];
      }
      for (int v = 0; v < 4; ++v) qc_all[(f * n1 + k) * 4 + v] = 0.5 * (qm[v] + qp[v]);
    }
  }
  if (visc) {
    broken_gradient<S>(L, e, qe, gb.data());
    for (int v = 0; v < 4; ++v)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          S qx = 0.0, qy = 0.0;
          for (int m = 0; m < n1; ++m) {
            qx += b.D[i * n1 + m] * qe[v * N + j * n1 + m];
            qy += b.D[j * n1 + m] * qe[v * N + m * n1 + i];
          }
          // xi faces 3 (xi = -1) and 1 (xi = +1) at face point j; eta faces
          // 0 (eta = -1) and 2 (eta = +1) at face point i.
          qx += b.gL[i] * (qc_all[(3 * n1 + j) * 4 + v] - qm_all[(3 * n1 + j) * 4 + v]) +
                b.gR[i] * (qc_all[(1 * n1 + j) * 4 + v] - qm_all[(1 * n1 + j) * 4 + v]);
          qy += b.gL[j] * (qc_all[(0 * n1 + i) * 4 + v] - qm_all[(0 * n1 + i) * 4 + v]) +
                b.gR[j] * (qc_all[(2 * n1 + i) * 4 + v] - qm_all[(2 * n1 + i) * 4 + v]);
          const double* mt = &L.g.met[((size_t)e * N + j * n1 + i) * 5];
          int pt = j * n1 + i;
          gc[(0 * 4 + v) * N + pt] = (mt[3] * qx - mt[2] * qy) / mt[4];
          gc[(1 * 4 + v) * N + pt] = (-mt[1] * qx + mt[0] * qy) / mt[4];
        }
  }
  for (int pt = 0; pt < N; ++pt) {
    const double* m = &L.g.met[((size_t)e * N + pt) * 5];
    S q[4] = {qe[0 * N + pt], qe[1 * N + pt], qe[2 * N + pt], qe[3 * N + pt]};
    S fx[4], fy[4];
    euler_flux_n(q, 1.0, 0.0, ph, fx);
    euler_flux_n(q, 0.0, 1.0, ph, fy);
    if (visc) {
      S d[8], fv[4], gv[4];
      for (int c = 0; c < 8; ++c) d[c] = gc[c * N + pt];
      viscous_flux(q, d, ph, fv, gv);
      for (int v = 0; v < 4; ++v) { fx[v] -= fv[v]; fy[v] -= gv[v]; }
    }
    for (int v = 0; v < 4; ++v) {
      Ft[v * N + pt] = m[3] * fx[v] - m[1] * fy[v];    //  y_eta f - x_eta g
      Gt[v * N + pt] = -m[2] * fx[v] + m[0] * fy[v];   // -y_xi f + x_xi g
    }
  }
  std::vector<S> acc(4 * N, S(0.0));
  for (int v = 0; v < 4; ++v)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        S s = 0.0;
        for (int m = 0; m < n1; ++m) s += b.D[i * n1 + m] * Ft[v * N + j * n1 + m];
        for (int m = 0; m < n1; ++m) s += b.D[j * n1 + m] * Gt[v * N + m * n1 + i];
        acc[v * N + j * n1 + i] = s;
      }
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < n1; ++k) {
      S qm[4], qp[4], fo[4];
      const bool bnd = o->nbr[(e * 4 + f) * 3 + 0] < 0;
      const int bc = o->nbr[(e * 4 + f) * 3 + 1];
      for (int v = 0; v < 4; ++v) qm[v] = qm_all[(f * n1 + k) * 4 + v];
      const double* t = &ntr[(((size_t)e * 4 + f) * n1 + k) * NT];
      for (int v = 0; v < 4; ++v) qp[v] = qp_all[(f * n1 + k) * 4 + v];
      const double* Sv = &L.g.fS[(((size_t)e * 4 + f) * n1 + k) * 2];
      roe_flux(qm, qp, Sv[0], Sv[1], ph, fo);
      if (visc) {
        // Common gradient, eq. com_grad_q: broken gradients of both sides
        // at the face point plus their BR2 liftings.
        double Jm = L.g.fJ[((size_t)e * 4 + f) * n1 + k], Jp = bnd ? Jm : t[12];
        S gm[8], gp[8], dcom[8], qcm[4], fv[4], gv[4];
        trace_state(b, gb.data(), N, f, k, gm);
        trace_state(b, gb.data() + 4 * N, N, f, k, gm + 4);
        for (int c = 0; c < 8; ++c) gp[c] = bnd ? gm[c] : S(t[4 + c]);
        for (int v = 0; v < 4; ++v) {
          S qcv = qc_all[(f * n1 + k) * 4 + v];
          qcm[v] = qcv;
          S rm = eta_f * gface * (qcv - qm[v]) / Jm;    // times S_out
          S rp = eta_f * gface * (qcv - qp[v]) / Jp;    // times -S_out
          dcom[v] = 0.5 * (gm[v] + gp[v] + (rm - rp) * Sv[0]);
          dcom[4 + v] = 0.5 * (gm[4 + v] + gp[4 + v] + (rm - rp) * Sv[1]);
        }
        viscous_flux(qcm, dcom, ph, fv, gv);
        const int nv = (bnd && bc != 4) ? 3 : 4;   // walls: no viscous energy flux
        for (int v = 0; v < nv; ++v) fo[v] -= fv[v] * Sv[0] + gv[v] * Sv[1];
      }
      double sg = (f == 1 || f == 2) ? 1.0 : -1.0;        // outward -> reference-direction
      const std::vector<double>& l = (f == 1 || f == 2) ? b.lp : b.lm;
      const std::vector<double>& gp = (f == 1 || f == 2) ? b.gR : b.gL;
      for (int v = 0; v < 4; ++v) {
        const std::vector<S>& Fl = (f == 1 || f == 3) ? Ft : Gt;
        S loc = 0.0;
        for (int m = 0; m < n1; ++m) loc += l[m] * Fl[v * N + line_pt(P, f, k, m)];
        S jump = sg * fo[v] - loc;
        for (int m = 0; m < n1; ++m) acc[v * N + line_pt(P, f, k, m)] += gp[m] * jump;
      }
    }
  for (int v = 0; v < 4; ++v)
    for (int pt = 0; pt < N; ++pt) {
      double J = L.g.met[((size_t)e * N + pt) * 5 + 4];
      Re[v * N + pt] = -acc[v * N + pt] / J;
    }
}

// Element loops below may run on several host threads (OpenMP, when the
// library is built with it and orc_set_threads asks for more than one): each
// element's result depends only on frozen inputs and is written to its own
// slots, so the results do not depend on the thread count.
static void full_residual(const Oracle* o, const Level& L, const double* q, double* R) {
  int N = L.g.N, E = o->E;
  std::vector<double> tr;
  neighbour_traces(o, L, q, tr);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int e = 0; e < E; ++e) {
    std::vector<double> qe(4 * N), Re(4 * N);
    for (int v = 0; v < 4; ++v)
      for (int p = 0; p < N; ++p) qe[v * N + p] = q[((size_t)v * E + e) * N + p];
    element_residual<double>(o, L, e, qe.data(), tr.data(), Re.data());
    for (int v = 0; v < 4; ++v)
      for (int p = 0; p < N; ++p) R[((size_t)v * E + e) * N + p] = Re[v * N + p];
  }
}

// Level system residual F_l(q) - S_l.  F follows eq. ESDIRK_primitive:
// F = -q_c(q)/(omega dt) + R(q) + src.  On the finest level src is the stage
// source; on coarser levels the state-independent source is dropped (reading:
// it cancels exactly between F_l(q) and S_l = F_l(q^b) + P d).
static void level_F(const Oracle* o, int l, const double* q, bool with_src, bool minus_S, double* F) {
  const Level& L = o->lev[l];
  int N = L.g.N, E = o->E;
  size_t tot = (size_t)4 * E * N;
  full_residual(o, L, q, F);
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qq[4], qc[4];
      for (int v = 0; v < 4; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
      cons_from_prim(qq, o->ph, qc);
      for (int v = 0; v < 4; ++v) {
        size_t id = ((size_t)v * E + e) * N + p;
        F[id] += -qc[v] / o->omega_dt;
        if (with_src) F[id] += o->src[id];
      }
    }
  if (minus_S)
    for (size_t i = 0; i < tot; ++i) F[i] -= L.S[i];
}

// Element block D_e = Gamma/dtau + M/(omega dt) - dR_e/dq_e
// (eq. linearized_pseudo_transient_final, block diagonal of eq.
// smoothing_element_jacobi).  dR_e/dq_e by complex step with neighbours frozen.
static void element_block(const Oracle* o, const Level& L, int e, const double* q,
                          const double* ntr, double dtau, double* Dm) {
  int N = L.g.N, n = 4 * N, E = o->E;
  const double h = 1e-30;
  std::vector<cplx> qe(n), Re(n);
  for (int col = 0; col < n; ++col) {
    for (int v = 0; v < 4; ++v)
      for (int p = 0; p < N; ++p) qe[v * N + p] = cplx(q[((size_t)v * E + e) * N + p], 0.0);
    qe[col] += cplx(0.0, h);
    element_residual<cplx>(o, L, e, qe.data(), ntr, Re.data());
    for (int row = 0; row < n; ++row) Dm[row * n + col] = -Re[row].imag() / h;
  }
  for (int p = 0; p < N; ++p) {
    double qq[4];
    for (int v = 0; v < 4; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
    double eps = precond_eps(qq, o->ph);
    double G[4][4], M[4][4];
    Gamma_matrix(qq, eps, o->ph, G);
    M_matrix(qq, o->ph, M);
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c)
        Dm[(a * N + p) * n + (c * N + p)] += G[a][c] / dtau + M[a][c] / o->omega_dt;
  }
}

static int refresh_level(Oracle* o, int l) {
  Level& L = o->lev[l];
  int N = L.g.N, n = 4 * N, E = o->E;
  std::vector<double> tr;
  neighbour_traces(o, L, L.q.data(), tr);
  L.lu.assign((size_t)E * n * n, 0.0);
  L.piv.assign((size_t)E * n, 0);
  int singular = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(| : singular)
#endif
  for (int e = 0; e < E; ++e) {
    double* Dm = &L.lu[(size_t)e * n * n];
    element_block(o, L, e, L.q.data(), tr.data(), o->dtau, Dm);
    if (!lu_factor(n, Dm, &L.piv[(size_t)e * n])) singular |= 1;
  }
  return singular ? -4 : 0;
}

// Element-Jacobi sweep, eq. smoothing_element_jacobi with alpha_r = 1.
static void smooth(Oracle* o, int l, int nsweep) {
  Level& L = o->lev[l];
  int N = L.g.N, n = 4 * N, E = o->E;
  L.F.resize((size_t)4 * E * N);
  for (int s = 0; s < nsweep; ++s) {
    level_F(o, l, L.q.data(), l == 0, l > 0, L.F.data());
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int e = 0; e < E; ++e) {
      std::vector<double> x(n);
      for (int v = 0; v < 4; ++v)
        for (int p = 0; p < N; ++p) x[v * N + p] = L.F[((size_t)v * E + e) * N + p];
      lu_solve(n, &L.lu[(size_t)e * n * n], &L.piv[(size_t)e * n], x.data());
      for (int v = 0; v < 4; ++v)
        for (int p = 0; p < N; ++p) L.q[((size_t)v * E + e) * N + p] += x[v * N + p];
    }
  }
}

static void apply_tensor(const std::vector<double>& op, int nout, int nin, int E,
                         const double* in, double* out) {
  // out[v][e][(j,i)] = sum_{a,b} op[i][a] op[j][b] in[v][e][(b,a)]
  int Nin = nin * nin, Nout = nout * nout;
  for (int v = 0; v < 4; ++v)
    for (int e = 0; e < E; ++e)
      for (int j = 0; j < nout; ++j)
        for (int i = 0; i < nout; ++i) {
          double s = 0.0;
          for (int bb = 0; bb < nin; ++bb)
            for (int a = 0; a < nin; ++a)
              s += op[i * nin + a] * op[j * nin + bb] * in[((size_t)v * E + e) * Nin + bb * nin + a];
          out[((size_t)v * E + e) * Nout + j * nout + i] = s;
        }
}

// One FAS V-cycle from level l down (Section 3): pre-smooth, defect,
// restrict state and defect, coarse forcing, recurse, prolong the
// correction, post-smooth.  The coarsest level smooths once.
static int vcycle_level(Oracle* o, int l, bool refresh) {
  Level& L = o->lev[l];
  int E = o->E;
  if (refresh) { int st = refresh_level(o, l); if (st) return st; }
  smooth(o, l, o->cfg.n_smooth[l]);
  if (l == o->cfg.n_levels - 1) return 0;
  Level& C = o->lev[l + 1];
  int Nf = L.g.N, Nc = C.g.N;
  std::vector<double> d((size_t)4 * E * Nf);
  level_F(o, l, L.q.data(), l == 0, l > 0, d.data());
  for (auto& x : d) x = -x;                                   // d = S - F(q^a)
  C.q.resize((size_t)4 * E * Nc);
  apply_tensor(o->Rm[l], C.g.P + 1, L.g.P + 1, E, L.q.data(), C.q.data());
  C.qb = C.q;
  std::vector<double> Pd((size_t)4 * E * Nc), Fc((size_t)4 * E * Nc);
  apply_tensor(o->Rm[l], C.g.P + 1, L.g.P + 1, E, d.data(), Pd.data());
  level_F(o, l + 1, C.q.data(), false, false, Fc.data());
  C.S.resize((size_t)4 * E * Nc);
  for (size_t i = 0; i < C.S.size(); ++i) C.S[i] = Fc[i] + Pd[i];
  int st = vcycle_level(o, l + 1, refresh);
  if (st) return st;
  std::vector<double> corr((size_t)4 * E * Nc), pc((size_t)4 * E * Nf);
  for (size_t i = 0; i < corr.size(); ++i) corr[i] = C.q[i] - C.qb[i];
  apply_tensor(o->Pm[l], L.g.P + 1, C.g.P + 1, E, corr.data(), pc.data());
  for (size_t i = 0; i < pc.size(); ++i) L.q[i] += pc[i];
  smooth(o, l, o->cfg.n_smooth[l]);
  return 0;
}

// ||F||_L2 of eq. ser and of the stopping test (Section 2.4).  The paper does
// not say how the equations are weighted.  Reading: each equation is divided
// by its reference scale (the caller passes the free-stream convective flux
// scales rho U, rho U^2, rho U^2, rho U H): at Ma = 0.005 the unweighted norm
// is the energy residual alone, H ~ 1/Ma^2 times any mass imbalance, and a
// stage that starts near its solution then stalls (the first element-Jacobi
// sweep raises it 350-fold while the scaled norm falls 60-fold).
static double residual_norm(const Oracle* o, const std::vector<double>& F) {
  size_t plane = F.size() / 4;
  double s = 0.0;
  for (int v = 0; v < 4; ++v) {
    double sc = o->cfg.res_scale[v] > 0.0 ? o->cfg.res_scale[v] : 1.0;
    double t = 0.0;
    for (size_t i = 0; i < plane; ++i) t += F[v * plane + i] * F[v * plane + i];
    s += t / (sc * sc);
  }
  return std::sqrt(s);
}

// ESDIRK3 tableau (Section 2.4 cites Bijl et al. 2002, which prints nothing):
// reading = the stiffly accurate, L-stable 4-stage third-order ESDIRK with
// c = (0, 2g, 3/5, 1), a_ii = g, last row = b, derived here from the order
// conditions.  g is the root in (0.4, 0.5) of g^3 - 3g^2 + 3g/2 - 1/6 = 0.
static void esdirk3_tableau(double A[6][6], double b[6], double c[6]) {
  double lo = 0.4, hi = 0.5;
  auto fpoly = [](double g) { return g * g * g - 3 * g * g + 1.5 * g - 1.0 / 6.0; };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if ((fpoly(lo) < 0) == (fpoly(mid) < 0)) lo = mid; else hi = mid;
  }
  double g = 0.5 * (lo + hi);
  for (int i = 0; i < 6; ++i) { b[i] = c[i] = 0.0; for (int j = 0; j < 6; ++j) A[i][j] = 0.0; }
  c[0] = 0.0; c[1] = 2 * g; c[2] = 0.6; c[3] = 1.0;
  // b1..b3 from sum b = 1, sum b c = 1/2, sum b c^2 = 1/3 with b4 = g, c4 = 1.
  double M3[9] = {1, 1, 1, c[0], c[1], c[2], c[0] * c[0], c[1] * c[1], c[2] * c[2]};
  double r3[3] = {1 - g, 0.5 - g, 1.0 / 3.0 - g};
  int piv[3];
  lu_factor(3, M3, piv);
  lu_solve(3, M3, piv, r3);
  b[0] = r3[0]; b[1] = r3[1]; b[2] = r3[2]; b[3] = g;
  A[1][0] = g; A[1][1] = g;
  // sum_i b_i (A c)_i = 1/6 fixes a32:  b2 (2g^2) + b3 (2 g a32 + 0.6 g) + b4 (1/2) = 1/6
  double a32 = (1.0 / 6.0 - b[1] * 2 * g * g - b[2] * 0.6 * g - b[3] * 0.5) / (b[2] * 2 * g);
  A[2][1] = a32; A[2][2] = g; A[2][0] = c[2] - g - a32;
  for (int j = 0; j < 4; ++j) A[3][j] = b[j];
}

// ESDIRK2 (Section 2.4 cites Kennedy & Carpenter 2016: second order, three
// stages): stiffly accurate, c = (0, 2g, 1), a_ii = g, last row = b.  The
// order conditions sum b = 1 and sum b c = 1/2 give b2 = (1/2 - g)/(2g),
// b1 = 1 - g - b2; L-stability (R(z) -> 0 as z -> -inf) fixes g = 1 - 1/sqrt 2.
static void esdirk2_tableau(double A[6][6], double b[6], double c[6]) {
  for (int i = 0; i < 6; ++i) { b[i] = c[i] = 0.0; for (int j = 0; j < 6; ++j) A[i][j] = 0.0; }
  const double g = 1.0 - 1.0 / std::sqrt(2.0);
  c[1] = 2 * g; c[2] = 1.0;
  b[2] = g;
  b[1] = (0.5 - g) / (2 * g);
  b[0] = 1.0 - g - b[1];
  A[1][0] = g; A[1][1] = g;
  for (int j = 0; j < 3; ++j) A[2][j] = b[j];
}

// ESDIRK4 (Section 2.4 cites Bijl et al. 2002: fourth order, six stages):
// reading = the implicit tableau of Kennedy & Carpenter's ARK4(3)6L[2]SA,
// taken as published (gamma = 1/4, stiffly accurate).  The tests check the
// eight fourth-order conditions and L-stability.
static void esdirk4_tableau(double A[6][6], double b[6], double c[6]) {
  for (int i = 0; i < 6; ++i) { b[i] = c[i] = 0.0; for (int j = 0; j < 6; ++j) A[i][j] = 0.0; }
  const double g = 0.25;
  const double cc[6] = {0.0, 0.5, 83.0 / 250.0, 31.0 / 50.0, 17.0 / 20.0, 1.0};
  const double bb[6] = {82889.0 / 524892.0, 0.0, 15625.0 / 83664.0, 69875.0 / 102672.0, -2260.0 / 8211.0, 0.25};
  for (int i = 0; i < 6; ++i) { c[i] = cc[i]; b[i] = bb[i]; }
  for (int i = 1; i < 6; ++i) A[i][i] = g;
  A[1][0] = g;
  A[2][0] = 8611.0 / 62500.0; A[2][1] = -1743.0 / 31250.0;
  A[3][0] = 5012029.0 / 34652500.0; A[3][1] = -654441.0 / 2922500.0; A[3][2] = 174375.0 / 388108.0;
  A[4][0] = 15267082809.0 / 155376265600.0; A[4][1] = -71443401.0 / 120774400.0;
  A[4][2] = 730878875.0 / 902184768.0; A[4][3] = 2285395.0 / 8070912.0;
  for (int j = 0; j < 6; ++j) A[5][j] = b[j];
}

// Scheme by number of stages: 3 -> ESDIRK2, 4 -> ESDIRK3, 6 -> ESDIRK4.
static int esdirk_tableau(int stages, double A[6][6], double b[6], double c[6]) {
  if (stages == 3) { esdirk2_tableau(A, b, c); return 3; }
  if (stages == 6) { esdirk4_tableau(A, b, c); return 6; }
  esdirk3_tableau(A, b, c);
  return 4;
}

extern "C" {

// Host threads of the element loops (OpenMP builds only; 1 otherwise).
// Returns the number of threads the loops will use.
int orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
  return n > 0 ? n : 1;
#else
  (void)n;
  return 1;
#endif
}

int orc_esdirk(int stages, double* A, double* b, double* c) {
  double AA[6][6], bb[6], cc[6];
  int s = esdirk_tableau(stages, AA, bb, cc);
  for (int i = 0; i < s; ++i) {
    b[i] = bb[i]; c[i] = cc[i];
    for (int j = 0; j < s; ++j) A[i * s + j] = AA[i][j];
  }
  return s;
}

int orc_basis(int P, double* x, double* w, double* D, double* lm, double* lp, double* gL, double* gR) {
  Basis1D b = make_basis(P);
  int n = P + 1;
  for (int i = 0; i < n; ++i) {
    x[i] = b.x[i]; w[i] = b.w[i]; lm[i] = b.lm[i]; lp[i] = b.lp[i]; gL[i] = b.gL[i]; gR[i] = b.gR[i];
  }
  for (int i = 0; i < n * n; ++i) D[i] = b.D[i];
  return 0;
}

int orc_transfer(int Pf, int Pc, double* Rop, double* Pop) {
  Basis1D f = make_basis(Pf), c = make_basis(Pc);
  std::vector<double> R = make_restriction(f, c), I = make_prolongation(f, c);
  memcpy(Rop, R.data(), sizeof(double) * R.size());
  memcpy(Pop, I.data(), sizeof(double) * I.size());
  return 0;
}

int orc_esdirk3(double* A, double* b, double* c) {
  double AA[6][6], bb[6], cc[6];
  esdirk3_tableau(AA, bb, cc);
  for (int i = 0; i < 4; ++i) {
    b[i] = bb[i]; c[i] = cc[i];
    for (int j = 0; j < 4; ++j) A[i * 4 + j] = AA[i][j];
  }
  return 0;
}

// Pointwise physics, exposed for the pins.
int orc_point_matrices(const double* q, double gamma, double Ma_inf, double kappa, int cutoff,
                       double* M, double* G, double* eps_out) {
  Phys ph = {gamma, Ma_inf, kappa, cutoff};
  double MM[4][4], GG[4][4];
  double e = precond_eps(q, ph);
  M_matrix(q, ph, MM);
  Gamma_matrix(q, e, ph, GG);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) { M[i * 4 + j] = MM[i][j]; G[i * 4 + j] = GG[i][j]; }
  *eps_out = e;
  return 0;
}

int orc_flux(const double* q, double nx, double ny, double gamma, double* f, double* A) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  euler_flux_n(q, nx, ny, ph, f);
  double AA[4][4];
  flux_jacobian_n(q, nx, ny, ph, AA);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i * 4 + j] = AA[i][j];
  return 0;
}

// Complex-step derivative of the flux, to pin the hand-written Jacobian.
int orc_flux_cs(const double* q, double nx, double ny, double gamma, double* A) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  for (int c = 0; c < 4; ++c) {
    cplx qq[4], f[4];
    for (int v = 0; v < 4; ++v) qq[v] = cplx(q[v], v == c ? 1e-30 : 0.0);
    euler_flux_n(qq, nx, ny, ph, f);
    for (int v = 0; v < 4; ++v) A[v * 4 + c] = f[v].imag() / 1e-30;
  }
  return 0;
}

int orc_roe(const double* qm, const double* qp, double Sx, double Sy, double gamma, double Ma_inf,
            double kappa, int cutoff, double* out) {
  Phys ph = {gamma, Ma_inf, kappa, cutoff};
  roe_flux(qm, qp, Sx, Sy, ph, out);
  return 0;
}

int orc_cons_from_prim(const double* q, double gamma, double* qc) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  cons_from_prim(q, ph, qc);
  return 0;
}

int orc_prim_from_cons(const double* qc, double gamma, double* q) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  prim_from_cons(qc, ph, q);
  return 0;
}

void* orc_create(const OrcConfig* cfg, int E, int Ng, const double* nodes, const int* nbr) {
  Oracle* o = new Oracle();
  o->cfg = *cfg;
  o->ph = {cfg->gamma, cfg->Ma_inf, cfg->kappa, cfg->cutoff};
  o->ph.mu = cfg->mu;
  o->ph.Pr = cfg->Pr;
  o->E = E; o->Ng = Ng;
  int nn = (Ng + 1) * (Ng + 1);
  o->nodes.assign(nodes, nodes + (size_t)E * nn * 2);
  o->nbr.assign(nbr, nbr + (size_t)E * 12);
  for (int i = 0; i < E * 4; ++i) {
    int en = nbr[i * 3], fn = nbr[i * 3 + 1];
    // slip walls are for inviscid runs only; a no-slip wall state has u = 0,
    // where eps = min(1, max(kappa Ma_inf, Ma)) needs the cut-off
    bool ok = en >= 0 ? (en < E && fn >= 0 && fn < 4)
                      : (en == -1 && fn >= 2 && fn <= 4 && !(fn == 2 && cfg->mu > 0) &&
                         !(fn == 3 && !(cfg->cutoff && cfg->kappa * cfg->Ma_inf > 0)));
    if (!ok) { delete o; return nullptr; }
  }
  o->dx.resize(E);
  for (int e = 0; e < E; ++e) o->dx[e] = element_dx(Ng, &o->nodes[(size_t)e * nn * 2]);
  o->lev.resize(cfg->n_levels);
  for (int l = 0; l < cfg->n_levels; ++l) {
    build_level_geom(o, cfg->P[l], &o->lev[l].g);
    size_t tot = (size_t)4 * E * o->lev[l].g.N;
    o->lev[l].q.assign(tot, 0.0);
    o->lev[l].S.assign(tot, 0.0);
  }
  for (int l = 0; l + 1 < cfg->n_levels; ++l) {
    o->Rm.push_back(make_restriction(o->lev[l].g.b, o->lev[l + 1].g.b));
    o->Pm.push_back(make_prolongation(o->lev[l].g.b, o->lev[l + 1].g.b));
  }
  o->s = esdirk_tableau(cfg->esdirk_stages, o->A, o->b, o->c);
  o->omega_dt = 1.0;
  o->dtau = cfg->dtau_init;
  o->src.assign((size_t)4 * E * o->lev[0].g.N, 0.0);
  return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

int orc_metrics(void* h, int level, double* met, double* fS) {
  Oracle* o = (Oracle*)h;
  const Level& L = o->lev[level];
  memcpy(met, L.g.met.data(), sizeof(double) * L.g.met.size());
  memcpy(fS, L.g.fS.data(), sizeof(double) * L.g.fS.size());
  return 0;
}

// Physical coordinates of the solution points of a level, (E, N, 2).
static double dtau_min(const Oracle* o, const double* q);

int orc_element_dx(void* h, double* dx) {
  Oracle* o = (Oracle*)h;
  for (int e = 0; e < o->E; ++e) dx[e] = o->dx[e];
  return 0;
}

double orc_dtau_min(void* h, const double* q) { return dtau_min((Oracle*)h, q); }

int orc_coords(void* h, int level, double* xy) {
  Oracle* o = (Oracle*)h;
  const Level& L = o->lev[level];
  int P = L.g.P, n1 = P + 1, N = L.g.N, Ng = o->Ng, nn = (Ng + 1) * (Ng + 1);
  std::vector<double> r(Ng + 1);
  for (int a = 0; a <= Ng; ++a) r[a] = -1.0 + 2.0 * a / Ng;
  for (int e = 0; e < o->E; ++e)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        double x = 0.0, y = 0.0;
        for (int b = 0; b <= Ng; ++b)
          for (int a = 0; a <= Ng; ++a) {
            double phi = lagrange(r, a, L.g.b.x[i]) * lagrange(r, b, L.g.b.x[j]);
            x += phi * o->nodes[((size_t)e * nn + b * (Ng + 1) + a) * 2 + 0];
            y += phi * o->nodes[((size_t)e * nn + b * (Ng + 1) + a) * 2 + 1];
          }
        xy[((size_t)e * N + j * n1 + i) * 2 + 0] = x;
        xy[((size_t)e * N + j * n1 + i) * 2 + 1] = y;
      }
  return 0;
}

int orc_residual(void* h, int level, const double* q, double* R) {
  Oracle* o = (Oracle*)h;
  full_residual(o, o->lev[level], q, R);
  return 0;
}

// Sets the stage data used by the level-0 system: src and omega*dt.
int orc_set_stage(void* h, const double* src, double omega_dt) {
  Oracle* o = (Oracle*)h;
  o->omega_dt = omega_dt;
  memcpy(o->src.data(), src, sizeof(double) * o->src.size());
  return 0;
}

// F_l(q) (with the stage source on level 0, without S).
int orc_stage_F(void* h, int level, const double* q, double* F) {
  Oracle* o = (Oracle*)h;
  level_F(o, level, q, level == 0, false, F);
  return 0;
}

// Full element blocks D_e (row-major n*n per element) of a level at state q.
int orc_blocks(void* h, int level, const double* q, double dtau, double* D) {
  Oracle* o = (Oracle*)h;
  const Level& L = o->lev[level];
  int n = 4 * L.g.N;
  std::vector<double> tr;
  neighbour_traces(o, L, q, tr);
  for (int e = 0; e < o->E; ++e) element_block(o, L, e, q, tr.data(), dtau, D + (size_t)e * n * n);
  return 0;
}

int orc_lu_solve(int n, const double* A, const double* rhs, double* x) {
  std::vector<double> a(A, A + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, a.data(), piv.data())) return -4;
  for (int i = 0; i < n; ++i) x[i] = rhs[i];
  lu_solve(n, a.data(), piv.data(), x);
  return 0;
}

int orc_restrict(void* h, int lf, const double* qf, double* qc) {
  Oracle* o = (Oracle*)h;
  apply_tensor(o->Rm[lf], o->lev[lf + 1].g.P + 1, o->lev[lf].g.P + 1, o->E, qf, qc);
  return 0;
}

int orc_prolong(void* h, int lf, const double* qc, double* qf) {
  Oracle* o = (Oracle*)h;
  apply_tensor(o->Pm[lf], o->lev[lf].g.P + 1, o->lev[lf + 1].g.P + 1, o->E, qc, qf);
  return 0;
}

// One V-cycle on the finest-level state q (in/out) with the current stage data.
int orc_vcycle(void* h, double* q, double dtau, int refresh) {
  Oracle* o = (Oracle*)h;
  Level& L = o->lev[0];
  memcpy(L.q.data(), q, sizeof(double) * L.q.size());
  std::fill(L.S.begin(), L.S.end(), 0.0);
  o->dtau = dtau;
  int st = vcycle_level(o, 0, refresh != 0);
  memcpy(q, L.q.data(), sizeof(double) * L.q.size());
  return st;
}

// dtau_min of the CFL definition (Section 2.4): the smaller of
// min_e (dx_e/(P+1)) / (c + |v|)_e and min_e (dx_e/(P+1))^2 / (mu/rho)_e on the
// finest level.  Reading: (c + |v|)_e is the largest and rho_e the smallest
// value over the element's solution points.
static double dtau_min(const Oracle* o, const double* q) {
  const Level& L = o->lev[0];
  int N = L.g.N, E = o->E, P = L.g.P;
  double best = 1e300;
  for (int e = 0; e < E; ++e) {
    double smax = 0.0, rmin = 1e300;
    for (int p = 0; p < N; ++p) {
      double pr = q[((size_t)0 * E + e) * N + p], u = q[((size_t)1 * E + e) * N + p];
      double v = q[((size_t)2 * E + e) * N + p], T = q[((size_t)3 * E + e) * N + p];
      smax = std::max(smax, std::sqrt(o->ph.gamma * T) + std::sqrt(u * u + v * v));
      rmin = std::min(rmin, pr / T);
    }
    double hP = o->dx[e] / (P + 1);
    best = std::min(best, hP / smax);
    if (o->ph.mu > 0.0) best = std::min(best, hP * hP * rmin / o->ph.mu);
  }
  return best;
}

// Pseudo-transient continuation of one implicit stage (Section 2.4): a
// V-cycle per pseudo-iteration, SER growth of dtau (eq. ser, exponent 1.5),
// smoother refresh at m = 0 and every refresh_every iterations while
// dtau < dtau_max, stop at ||F^m|| <= tol ||F^0|| (unweighted 2-norm over all
// finest points and equations, evaluated at the start of each V-cycle).
// SER growth of eq. ser with the pseudo time step in place of the CFL
// number (dtau set directly, Section 4.1): fixed exponent 1.5, no lower clamp.
static double ser_next(double dtau, double prev_norm, double norm, double dtau_max) {
  return std::min(dtau * std::pow(prev_norm / norm, 1.5), dtau_max);
}

// Smoother refresh rule (Sections 4.1, 4.4): at the first pseudo-iteration
// of a stage, then every k-th one until the smoother has been built with
// dtau = dtau_max; after that it is no longer updated.  Reading: "if
// dtau = dtau_max the smoother is not updated anymore" refers to a smoother
// already built at dtau_max (taken literally, a dtau that reaches dtau_max
// within the first k iterations would freeze the smoother at dtau_init).
static bool refresh_due(int m, int k, double dtau_last_refresh, double dtau_max, bool always = false) {
  if (always) return m % k == 0;   // Section 4.1: every k-th pseudo-iteration
  return m == 0 || (m % k == 0 && dtau_last_refresh < dtau_max);
}

// Pseudo-transient continuation of one implicit stage (Section 2.4): a
// V-cycle per pseudo-iteration, SER growth of dtau, smoother refresh per
// refresh_due, stop at ||F^m|| <= tol ||F^0|| (residual_norm over all
// finest points, evaluated at the start of each V-cycle).
static int stage_solve(Oracle* o, double* q, int* iters, double* drop, double* norms_out, int max_norms) {
  Level& L = o->lev[0];
  size_t tot = L.q.size();
  std::vector<double> F(tot);
  double dtau_init = o->cfg.dtau_init, dtau_max = o->cfg.dtau_max;
  if (o->cfg.cfl_mode) {   // eq. CFL: dtau = CFL dtau_min, SER acting on the CFL number
    double dm = dtau_min(o, q);
    dtau_init = o->cfg.cfl_init * dm;
    dtau_max = o->cfg.cfl_max * dm;
  }
  double dtau = dtau_init, n0 = 0.0, prev = 0.0, dtau_built = 0.0;
  for (int m = 0;; ++m) {
    level_F(o, 0, q, true, false, F.data());
    double nm = residual_norm(o, F);
    if (norms_out && m < max_norms) norms_out[m] = nm;
    if (m == 0) n0 = nm;
    if (nm <= o->cfg.tol * n0 || n0 == 0.0) { *iters = m; *drop = n0 > 0 ? nm / n0 : 0.0; return 0; }
    if (!std::isfinite(nm)) { *iters = m; *drop = nm; return -5; }
    if (m >= o->cfg.max_pseudo) { *iters = m; *drop = nm / n0; return -6; }
    if (m > 0) dtau = ser_next(dtau, prev, nm, dtau_max);
    bool refresh = refresh_due(m, o->cfg.refresh_every, dtau_built, dtau_max, o->cfg.refresh_always != 0);
    if (refresh) dtau_built = dtau;
    int st = orc_vcycle(o, q, dtau, refresh);
    if (st) return st;
    prev = nm;
  }
}

// The dtau / refresh schedule stage_solve follows for a given norm sequence.
int orc_ser_schedule(const double* norms, int n, double dtau_init, double dtau_max, int k,
                     double* dtau_out, int* refresh_out) {
  double dtau = dtau_init, built = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m > 0) dtau = ser_next(dtau, norms[m - 1], norms[m], dtau_max);
    dtau_out[m] = dtau;
    refresh_out[m] = refresh_due(m, k, built, dtau_max) ? 1 : 0;
    if (refresh_out[m]) built = dtau;
  }
  return 0;
}

int orc_stage_solve(void* h, double* q, int* iters, double* drop, double* norms, int max_norms) {
  return stage_solve((Oracle*)h, q, iters, drop, norms, max_norms);
}

// One ESDIRK3 physical step (eq. ESDIRK_ns with the stage systems of eq.
// ESDIRK_primitive); stage initial guess q^{i,0} = q^{i-1} (reading).
int orc_esdirk_step(void* h, double* q, double dt, int* iters, double* drops) {
  Oracle* o = (Oracle*)h;
  Level& L = o->lev[0];
  int E = o->E, N = L.g.N;
  size_t tot = (size_t)4 * E * N;
  int s = o->s;
  std::vector<double> qcn(tot), qi(q, q + tot);
  std::vector<std::vector<double>> Rs(s, std::vector<double>(tot));
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qq[4], qc[4];
      for (int v = 0; v < 4; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
      cons_from_prim(qq, o->ph, qc);
      for (int v = 0; v < 4; ++v) qcn[((size_t)v * E + e) * N + p] = qc[v];
    }
  full_residual(o, L, qi.data(), Rs[0].data());
  double omega = o->A[1][1];
  o->omega_dt = omega * dt;
  for (int i = 1; i < s; ++i) {
    for (size_t k = 0; k < tot; ++k) {
      double acc = qcn[k];
      for (int j = 0; j < i; ++j) acc += dt * o->A[i][j] * Rs[j][k];
      o->src[k] = acc / o->omega_dt;
    }
    int st = stage_solve(o, qi.data(), &iters[i - 1], &drops[i - 1], nullptr, 0);
    if (st) return st;
    full_residual(o, L, qi.data(), Rs[i].data());
  }
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qc[4], qq[4];
      for (int v = 0; v < 4; ++v) {
        size_t k = ((size_t)v * E + e) * N + p;
        double acc = qcn[k];
        for (int i = 0; i < s; ++i) acc += dt * o->b[i] * Rs[i][k];
        qc[v] = acc;
      }
      prim_from_cons(qc, o->ph, qq);
      for (int v = 0; v < 4; ++v) q[((size_t)v * E + e) * N + p] = qq[v];
    }
  return 0;
}

}  // extern "C"

// ===========================================================================
// Three dimensions: hexahedral elements, 5 working variables
// q_p = (p, u, v, w, T) (Sections 2.1-2.4 with d = 3; Section 3).
//
// Layout conventions (shared with the CUDA library only through its C
// interface):
//   solution point (i, j, k) of a degree-P hexahedron has index
//   (k*(P+1) + j)*(P+1) + i, i along xi, j along eta, k along zeta;
//   a state array is variable-major: q[(v*E + e)*N + pt], N = (P+1)^3;
//   faces: f = 2*d + s, d = 0 (xi), 1 (eta), 2 (zeta), s = 0 (-1 side) or 1
//   (+1 side); a face point (a, b) has index b*(P+1) + a, a along the first
//   and b along the second of the other two reference directions in
//   increasing order (xi faces: (eta, zeta); eta faces: (xi, zeta); zeta
//   faces: (xi, eta));
//   nbr[(e*6+f)*3 + {0,1,2}] = (neighbour element, neighbour face,
//   orientation o); the neighbour's face point of (a, b) is (a', b') with
//   (s, t) = (o & 4) ? (b, a) : (a, b), a' = (o & 1) ? P - s : s,
//   b' = (o & 2) ? P - t : t; a boundary face has neighbour -1 and the
//   boundary type in the second slot (2 slip wall, 4 far field);
//   element geometry: (Ng+1)^3 Lagrange nodes at equispaced reference
//   positions, node (c*(Ng+1) + b)*(Ng+1) + a, a along xi;
//   nodes[(e*(Ng+1)^3 + node)*3 + {x, y, z}].
//
// Metric terms.  On curved hexahedra the metric terms J grad(xi^i) taken
// from the mapping at the solution points do not satisfy the discrete
// metric identity, so uniform flow is not steady.  Reading (the paper is
// silent): the conservative curl form, J a^i_n = -e_i . curl_xi(I(X_l grad_xi
// X_m)) with (n, m, l) cyclic, where I interpolates at the Gauss-Lobatto
// points of degree Pg = max(P, Ng, 1).  On a face the normal component
// involves only the face's own Gauss-Lobatto values, so both elements of a
// face see the same normal; with Pg >= Ng the interpolated gradient of the
// map is exact, its curl vanishes, and the normal does not change when an
// element is translated (periodic images of a face agree).  For P >= Ng
// these metric terms are polynomials of degree <= P in every direction, their
// discrete divergence at the Gauss solution points vanishes and uniform flow
// is exactly steady; below the geometry order (coarse P-levels of curved
// meshes) the scheme stays conservative and free-stream preservation holds
// to the interpolation error, as with the analytic metrics of the 2D
// elements.  The surface normal of a face point is the outward J a^d of the
// polynomial; |J| at the solution points is the determinant of the exact map.
// ===========================================================================

// Gauss-Lobatto points of degree n (n + 1 points): -1, the roots of L_n', +1.
static std::vector<double> gll_nodes(int n) {
  std::vector<double> x(n + 1);
  x[0] = -1.0; x[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    // Newton on L_n' from the Chebyshev-Gauss-Lobatto guess; L_n'' from
    // the Legendre equation (1 - t^2) L'' = 2 t L' - n (n+1) L.
    double t = -std::cos(M_PI * i / n);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(n, t, &L, &dL);
      double d2 = (2.0 * t * dL - n * (n + 1.0) * L) / (1.0 - t * t);
      double dt = dL / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  return x;
}

// ---- thermodynamics and preconditioning in 3D (Sections 2.1-2.2)
template <class S> static void cons_from_prim3(const S q[5], const Phys& ph, S qc[5]) {
  S rho = q[0] / q[4];
  S E = q[4] / (ph.gamma - 1.0) + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  qc[0] = rho; qc[1] = rho * q[1]; qc[2] = rho * q[2]; qc[3] = rho * q[3]; qc[4] = rho * E;
}

static void prim_from_cons3(const double qc[5], const Phys& ph, double q[5]) {
  double rho = qc[0], u = qc[1] / rho, v = qc[2] / rho, w = qc[3] / rho;
  double p = (ph.gamma - 1.0) * (qc[4] - 0.5 * rho * (u * u + v * v + w * w));
  q[0] = p; q[1] = u; q[2] = v; q[3] = w; q[4] = p / rho;
}

// M = dq_c/dq_p (Section 2.2, d = 3).
template <class S> static void M_matrix3(const S q[5], const Phys& ph, S M[5][5]) {
  S p = q[0], T = q[4];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M[i][j] = 0.0;
  M[0][0] = rp; M[0][4] = rT;
  for (int c = 1; c <= 3; ++c) { M[c][0] = rp * q[c]; M[c][c] = rho; M[c][4] = rT * q[c]; }
  M[4][0] = rp * H - 1.0;
  for (int c = 1; c <= 3; ++c) M[4][c] = rho * q[c];
  M[4][4] = rT * H + rho * Cp;
}

// eps of eq. eps_nonmove with |v| over three components.
template <class S> static S precond_eps3(const S q[5], const Phys& ph) {
  S Ma = cs_sqrt((q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / (ph.gamma * q[4]));
  S e = ph.cutoff ? cs_max(S(ph.kappa * ph.Ma_inf), Ma) : Ma;
  return cs_min(S(1.0), e);
}

// Gamma of eq. preconditioning: M with the first column rho_p replaced by
// Theta of eq. theta (U_r = eps c).
template <class S> static void Gamma_matrix3(const S q[5], const S& eps, const Phys& ph, S G[5][5]) {
  M_matrix3(q, ph, G);
  S T = q[4], rho = q[0] / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S Th = 1.0 / (eps * eps * ph.gamma * T) - rT / (rho * Cp);
  G[0][0] = Th;
  for (int c = 1; c <= 3; ++c) G[c][0] = Th * q[c];
  G[4][0] = Th * H - 1.0;
}

// Inviscid flux through the (possibly unnormalised) vector n (Section 2.1).
template <class S> static void euler_flux3(const S q[5], const double n[3], const Phys& ph, S f[5]) {
  S p = q[0], T = q[4];
  S rho = p / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S un = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  f[0] = rho * un;
  for (int c = 0; c < 3; ++c) f[1 + c] = rho * un * q[1 + c] + p * n[c];
  f[4] = rho * un * H;
}

// A_n = d f_n / d q_p, by hand from euler_flux3.
template <class S> static void flux_jacobian3(const S q[5], const double n[3], const Phys& ph, S A[5][5]) {
  S p = q[0], T = q[4];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S H = Cp * T + 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S un = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  A[0][0] = rp * un;
  for (int c = 0; c < 3; ++c) A[0][1 + c] = rho * n[c];
  A[0][4] = rT * un;
  for (int r = 0; r < 3; ++r) {
    A[1 + r][0] = rp * un * q[1 + r] + n[r];
    for (int c = 0; c < 3; ++c) A[1 + r][1 + c] = rho * q[1 + r] * n[c] + (r == c ? rho * un : S(0.0));
    A[1 + r][4] = rT * un * q[1 + r];
  }
  A[4][0] = rp * un * H;
  for (int c = 0; c < 3; ++c) A[4][1 + c] = rho * n[c] * H + rho * un * q[1 + c];
  A[4][4] = rT * un * H + rho * un * Cp;
}

// Solve G X = A (n x n, n <= 5) by elimination with partial pivoting on the real part.
template <class S> static void solve5(S G[5][5], S A[5][5], S X[5][5]) {
  S a[5][10];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) { a[i][j] = G[i][j]; a[i][5 + j] = A[i][j]; }
  for (int k = 0; k < 5; ++k) {
    int p = k;
    for (int i = k + 1; i < 5; ++i)
      if (std::fabs(re(a[i][k])) > std::fabs(re(a[p][k]))) p = i;
    if (p != k) for (int j = 0; j < 10; ++j) std::swap(a[k][j], a[p][j]);
    for (int i = k + 1; i < 5; ++i) {
      S l = a[i][k] / a[k][k];
      for (int j = k; j < 10; ++j) a[i][j] -= l * a[k][j];
    }
  }
  for (int c = 0; c < 5; ++c)
    for (int i = 4; i >= 0; --i) {
      S s = a[i][5 + c];
      for (int j = i + 1; j < 5; ++j) s -= a[i][j] * X[j][c];
      X[i][c] = s / a[i][i];
    }
}

// Preconditioned Roe flux of eq. invis_com in 3D, through the area-scaled
// normal Sv from - to +: the same construction as roe_flux (arithmetic mean of
// the primitive states, no entropy fix, Sylvester's formula over the three
// distinct eigenvalues u_n (three-fold), u_n' +- c' of eq. eigenvalues_para).
template <class S>
static void roe_flux3(const S qm[5], const S qp[5], const double Sv[3], const Phys& ph, S out[5]) {
  double dS = std::sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
  double n[3] = {Sv[0] / dS, Sv[1] / dS, Sv[2] / dS};
  S qa[5];
  for (int k = 0; k < 5; ++k) qa[k] = 0.5 * (qm[k] + qp[k]);
  S eps = precond_eps3(qa, ph);
  S G[5][5], A[5][5], Mt[5][5];
  Gamma_matrix3(qa, eps, ph, G);
  flux_jacobian3(qa, n, ph, A);
  solve5(G, A, Mt);
  S p = qa[0], T = qa[4];
  S rho = p / T, rp = 1.0 / T, rT = -rho / T;
  double Cp = ph.gamma / (ph.gamma - 1.0);
  S c = cs_sqrt(ph.gamma * T);
  S Ur = eps * c;
  S un = qa[1] * n[0] + qa[2] * n[1] + qa[3] * n[2];
  S beta = rp + rT / (rho * Cp);
  S alpha = 0.5 * (1.0 - beta * Ur * Ur);
  S cpr = cs_sqrt(alpha * alpha * un * un + Ur * Ur);
  S unp = un * (1.0 - alpha);
  S lam[3] = {un, unp + cpr, unp - cpr};
  S absM[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) absM[i][j] = 0.0;
  for (int k = 0; k < 3; ++k) {
    S Pk[5][5];
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) Pk[i][j] = (i == j) ? S(1.0) : S(0.0);
    for (int jj = 0; jj < 3; ++jj) {
      if (jj == k) continue;
      S fac[5][5], tmp[5][5];
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j)
          fac[i][j] = (Mt[i][j] - (i == j ? lam[jj] : S(0.0))) / (lam[k] - lam[jj]);
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
          S s = 0.0;
          for (int m = 0; m < 5; ++m) s += Pk[i][m] * fac[m][j];
          tmp[i][j] = s;
        }
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Pk[i][j] = tmp[i][j];
    }
    S al = cs_abs(lam[k]);
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) absM[i][j] += al * Pk[i][j];
  }
  S dq[5], t1[5], diss[5];
  for (int k = 0; k < 5; ++k) dq[k] = qp[k] - qm[k];
  for (int i = 0; i < 5; ++i) {
    S s = 0.0;
    for (int j = 0; j < 5; ++j) s += absM[i][j] * dq[j];
    t1[i] = s;
  }
  for (int i = 0; i < 5; ++i) {
    S s = 0.0;
    for (int j = 0; j < 5; ++j) s += G[i][j] * t1[j];
    diss[i] = s;
  }
  S fm[5], fp[5];
  euler_flux3(qm, n, ph, fm);
  euler_flux3(qp, n, ph, fp);
  for (int k = 0; k < 5; ++k) out[k] = (0.5 * (fm[k] + fp[k]) - 0.5 * diss[k]) * dS;
}

// Boundary ghost states in 3D (reading, as in 2D): slip wall (p, u - 2 u_n n, T),
// no-slip adiabatic wall (p, -u, T), far field the free stream.  n is the
// unit outward normal.
template <class S>
static void ghost_state3(int bc, const S qm[5], const double n[3], const double qinf[5], S qg[5]) {
  if (bc == 4) {
    for (int v = 0; v < 5; ++v) qg[v] = qinf[v];
    return;
  }
  qg[0] = qm[0]; qg[4] = qm[4];
  if (bc == 3) {
    for (int c = 0; c < 3; ++c) qg[1 + c] = -qm[1 + c];
    return;
  }
  S un = qm[1] * n[0] + qm[2] * n[1] + qm[3] * n[2];
  for (int c = 0; c < 3; ++c) qg[1 + c] = qm[1 + c] - 2.0 * un * n[c];
}

// Viscous fluxes in 3D (Section 2.1) from the state and the gradients
// d[c*5 + v] = d q_v / d x_c (q = (p, u, v, w, T)): stress tau_ij =
// mu (du_i/dx_j + du_j/dx_i - 2/3 div u delta_ij), heat conduction
// (mu Cp / Pr) dT/dx_j; fv[c*5 + v] is the flux of variable v in direction c:
// (0, tau_1c, tau_2c, tau_3c, u_i tau_ic + (mu Cp / Pr) dT/dx_c).
template <class S>
static void viscous_flux3(const S q[5], const S d[15], const Phys& ph, S fv[15]) {
  const double Cp = ph.gamma / (ph.gamma - 1.0), k = ph.mu * Cp / ph.Pr;
  S g[3][3];   // g[i][c] = d u_i / d x_c
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) g[i][c] = d[c * 5 + 1 + i];
  const S dv = g[0][0] + g[1][1] + g[2][2];
  for (int c = 0; c < 3; ++c) {
    S tau[3];
    for (int i = 0; i < 3; ++i) {
      tau[i] = ph.mu * (g[i][c] + g[c][i]);
      if (i == c) tau[i] -= ph.mu * (2.0 / 3.0) * dv;
    }
    fv[c * 5 + 0] = 0.0;
    for (int i = 0; i < 3; ++i) fv[c * 5 + 1 + i] = tau[i];
    fv[c * 5 + 4] = q[1] * tau[0] + q[2] * tau[1] + q[3] * tau[2] + k * d[c * 5 + 4];
  }
}

// ---- geometry of a hexahedron
static void map3(int Ng, const double* xn, const double r[3], double X[3], double dX[3][3]) {
  std::vector<double> g(Ng + 1);
  for (int a = 0; a <= Ng; ++a) g[a] = -1.0 + 2.0 * a / (Ng > 0 ? Ng : 1);
  for (int n = 0; n < 3; ++n) { X[n] = 0.0; dX[n][0] = dX[n][1] = dX[n][2] = 0.0; }
  for (int c = 0; c <= Ng; ++c)
    for (int b = 0; b <= Ng; ++b)
      for (int a = 0; a <= Ng; ++a) {
        double la = lagrange(g, a, r[0]), lb = lagrange(g, b, r[1]), lc = lagrange(g, c, r[2]);
        double da = lagrange_deriv(g, a, r[0]), db = lagrange_deriv(g, b, r[1]), dc = lagrange_deriv(g, c, r[2]);
        const double* Xn = xn + ((c * (Ng + 1) + b) * (Ng + 1) + a) * 3;
        for (int n = 0; n < 3; ++n) {
          X[n] += la * lb * lc * Xn[n];
          dX[n][0] += da * lb * lc * Xn[n];
          dX[n][1] += la * db * lc * Xn[n];
          dX[n][2] += la * lb * dc * Xn[n];
        }
      }
}

struct LevelGeom3 {
  int P, n1, N, NF;          // NF = (P+1)^2 points per face
  Basis1D b;
  std::vector<double> Ja;    // (e, pt, i, n): J a^i_n at the solution points
  std::vector<double> J;     // (e, pt)
  std::vector<double> xyz;   // (e, pt, 3)
  std::vector<double> fS;    // (e, face, fp, 3): outward area-scaled normal
  std::vector<double> fJ;    // (e, face, fp): |J| of the map at the face point
};

// Reference coordinates of face point (a, b) of face f.
static void face_ref(const Basis1D& b, int f, int a, int bb, double r[3]) {
  int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  r[d] = (f & 1) ? 1.0 : -1.0;
  r[t1] = b.x[a];
  r[t2] = b.x[bb];
}

// Solution point on the line normal to face f through face point (a, b), at
// position m along that line.
static inline int line_pt3(int P, int f, int a, int bb, int m) {
  int n1 = P + 1, d = f / 2, idx[3];
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  idx[d] = m; idx[t1] = a; idx[t2] = bb;
  return (idx[2] * n1 + idx[1]) * n1 + idx[0];
}

// Neighbour's face point of (a, b) under orientation o.
static inline void face_map3(int o, int P, int a, int bb, int* a2, int* b2) {
  int s = (o & 4) ? bb : a, t = (o & 4) ? a : bb;
  *a2 = (o & 1) ? P - s : s;
  *b2 = (o & 2) ? P - t : t;
}

// Conservative-curl metric terms J a^i_n of one element at reference point r:
// -(d_j W^n_k - d_k W^n_j), (i, j, k) cyclic, W^n_k = X_l dX_m/dxi_k with
// (n, m, l) cyclic, interpolated at the Gauss-Lobatto points gl.
static void curl_metrics(const std::vector<double>& gl, const std::vector<double>& W, const double r[3],
                         double Ja[3][3]) {
  const int ng = (int)gl.size();
  std::vector<double> l[3], dl[3];
  for (int d = 0; d < 3; ++d) {
    l[d].resize(ng); dl[d].resize(ng);
    for (int a = 0; a < ng; ++a) { l[d][a] = lagrange(gl, a, r[d]); dl[d][a] = lagrange_deriv(gl, a, r[d]); }
  }
  // dW[n][k][j] = d_j W^n_k at r
  double dW[3][3][3] = {};
  for (int c = 0; c < ng; ++c)
    for (int b = 0; b < ng; ++b)
      for (int a = 0; a < ng; ++a) {
        const double* w = &W[(size_t)((c * ng + b) * ng + a) * 9];
        double g0 = dl[0][a] * l[1][b] * l[2][c], g1 = l[0][a] * dl[1][b] * l[2][c], g2 = l[0][a] * l[1][b] * dl[2][c];
        for (int n = 0; n < 3; ++n)
          for (int k = 0; k < 3; ++k) {
            dW[n][k][0] += g0 * w[n * 3 + k];
            dW[n][k][1] += g1 * w[n * 3 + k];
            dW[n][k][2] += g2 * w[n * 3 + k];
          }
      }
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    for (int n = 0; n < 3; ++n) Ja[i][n] = -(dW[n][k][j] - dW[n][j][k]);
  }
}

struct OrcConfig3 {
  int n_levels;
  int P[8];
  int n_smooth[8];
  double gamma, Ma_inf, kappa;
  int cutoff;
  int esdirk_stages;
  double dtau_init, dtau_max, tol;
  int refresh_every, max_pseudo;
  double res_scale[5];
  double q_inf[5];
  int refresh_always;
  double mu, Pr;   // constant dynamic viscosity (0: Euler) and Prandtl number
};

struct Level3 {
  LevelGeom3 g;
  std::vector<double> q, qb, S, F;
  std::vector<double> lu;
  std::vector<int> piv;
};

struct Oracle3 {
  OrcConfig3 cfg;
  Phys ph;
  int E, Ng;
  std::vector<double> nodes;
  std::vector<int> nbr;
  std::vector<Level3> lev;
  std::vector<std::vector<double>> Rm, Pm;
  std::vector<double> src;
  double omega_dt, dtau;
  double A[6][6], b[6], c[6];
  int s;
};

static void build_level_geom3(Oracle3* o, int P, LevelGeom3* g) {
  g->P = P; g->n1 = P + 1; g->N = g->n1 * g->n1 * g->n1; g->NF = g->n1 * g->n1;
  g->b = make_basis(P);
  const int n1 = g->n1, E = o->E, Ng = o->Ng, nn = (Ng + 1) * (Ng + 1) * (Ng + 1);
  const int Pg = std::max(std::max(P, Ng), 1);
  const std::vector<double> gl = gll_nodes(Pg);
  const int ng = (int)gl.size();
  g->Ja.assign((size_t)E * g->N * 9, 0.0);
  g->J.assign((size_t)E * g->N, 0.0);
  g->xyz.assign((size_t)E * g->N * 3, 0.0);
  g->fS.assign((size_t)E * 6 * g->NF * 3, 0.0);
  g->fJ.assign((size_t)E * 6 * g->NF, 0.0);
  for (int e = 0; e < E; ++e) {
    const double* xn = &o->nodes[(size_t)e * nn * 3];
    // W^n_k = X_l dX_m/dxi_k at the Gauss-Lobatto points, (n, m, l) cyclic
    std::vector<double> W((size_t)ng * ng * ng * 9);
    for (int c = 0; c < ng; ++c)
      for (int b = 0; b < ng; ++b)
        for (int a = 0; a < ng; ++a) {
          double r[3] = {gl[a], gl[b], gl[c]}, X[3], dX[3][3];
          map3(Ng, xn, r, X, dX);
          double* w = &W[(size_t)((c * ng + b) * ng + a) * 9];
          for (int n = 0; n < 3; ++n) {
            int m = (n + 1) % 3, l = (n + 2) % 3;
            for (int k = 0; k < 3; ++k) w[n * 3 + k] = X[l] * dX[m][k];
          }
        }
    for (int kk = 0; kk < n1; ++kk)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          int pt = (kk * n1 + j) * n1 + i;
          double r[3] = {g->b.x[i], g->b.x[j], g->b.x[kk]}, X[3], dX[3][3], Ja[3][3];
          map3(Ng, xn, r, X, dX);
          curl_metrics(gl, W, r, Ja);
          for (int ii = 0; ii < 3; ++ii)
            for (int n = 0; n < 3; ++n) g->Ja[((size_t)e * g->N + pt) * 9 + ii * 3 + n] = Ja[ii][n];
          g->J[(size_t)e * g->N + pt] = dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
                                        dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
                                        dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
          for (int n = 0; n < 3; ++n) g->xyz[((size_t)e * g->N + pt) * 3 + n] = X[n];
        }
    for (int f = 0; f < 6; ++f)
      for (int bb = 0; bb < n1; ++bb)
        for (int a = 0; a < n1; ++a) {
          double r[3], Ja[3][3], X[3], dX[3][3];
          face_ref(g->b, f, a, bb, r);
          curl_metrics(gl, W, r, Ja);
          const double sg = (f & 1) ? 1.0 : -1.0;
          double* s = &g->fS[(((size_t)e * 6 + f) * g->NF + bb * n1 + a) * 3];
          for (int n = 0; n < 3; ++n) s[n] = sg * Ja[f / 2][n];
          map3(Ng, xn, r, X, dX);
          g->fJ[((size_t)e * 6 + f) * g->NF + bb * n1 + a] =
              dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
              dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
              dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
        }
  }
}

template <class S>
static void trace_state3(const Basis1D& b, const S* qe, int N, int f, int a, int bb, S out[5]) {
  int n1 = b.P + 1;
  const std::vector<double>& l = (f & 1) ? b.lp : b.lm;
  for (int v = 0; v < 5; ++v) {
    S s = 0.0;
    for (int m = 0; m < n1; ++m) s += l[m] * qe[v * N + line_pt3(b.P, f, a, bb, m)];
    out[v] = s;
  }
}

// Broken (uncorrected) gradient of one hexahedron's state at its solution
// points: reference derivatives by the Lagrange derivative matrix, then the
// chain rule grad q = (1/|J|) sum_i (J a^i) dq/dxi_i with the element's metric
// terms.  g[(c*5 + v)*N + pt], c = x, y, z.
template <class S>
static void broken_gradient3(const Level3& L, int e, const S* qe, S* g) {
  const Basis1D& b = L.g.b;
  const int n1 = L.g.n1, N = L.g.N;
  for (int v = 0; v < 5; ++v)
    for (int kk = 0; kk < n1; ++kk)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          const int pt = (kk * n1 + j) * n1 + i;
          S dr[3] = {0.0, 0.0, 0.0};
          for (int m = 0; m < n1; ++m) {
            dr[0] += b.D[i * n1 + m] * qe[v * N + (kk * n1 + j) * n1 + m];
            dr[1] += b.D[j * n1 + m] * qe[v * N + (kk * n1 + m) * n1 + i];
            dr[2] += b.D[kk * n1 + m] * qe[v * N + (m * n1 + j) * n1 + i];
          }
          const double* ja = &L.g.Ja[((size_t)e * N + pt) * 9];
          const double J = L.g.J[(size_t)e * N + pt];
          for (int c = 0; c < 3; ++c)
            g[(c * 5 + v) * N + pt] = (ja[0 * 3 + c] * dr[0] + ja[1 * 3 + c] * dr[1] + ja[2 * 3 + c] * dr[2]) / J;
        }
}

// Frozen neighbour data at every element face point, NT3 values each: the
// neighbour's state trace (5), with mu > 0 its broken-gradient trace (15,
// x, y, z per variable) and its |J| at that face point.
static const int NT3 = 21;

static void neighbour_traces3(const Oracle3* o, const Level3& L, const double* q, std::vector<double>& tr) {
  const int E = o->E, N = L.g.N, n1 = L.g.n1, NF = L.g.NF, P = L.g.P;
  const bool visc = o->ph.mu > 0.0;
  tr.assign((size_t)E * 6 * NF * NT3, 0.0);
  std::vector<double> qe(5 * N), g(15 * N);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int en = o->nbr[(e * 6 + f) * 3], fn = o->nbr[(e * 6 + f) * 3 + 1], or_ = o->nbr[(e * 6 + f) * 3 + 2];
      if (en < 0) continue;
      for (int v = 0; v < 5; ++v)
        for (int p = 0; p < N; ++p) qe[v * N + p] = q[((size_t)v * E + en) * N + p];
      if (visc) broken_gradient3<double>(L, en, qe.data(), g.data());
      for (int bb = 0; bb < n1; ++bb)
        for (int a = 0; a < n1; ++a) {
          int a2, b2;
          face_map3(or_, P, a, bb, &a2, &b2);
          double* t = &tr[(((size_t)e * 6 + f) * NF + bb * n1 + a) * NT3];
          trace_state3<double>(L.g.b, qe.data(), N, fn, a2, b2, t);
          if (visc) {
            for (int c = 0; c < 3; ++c) trace_state3<double>(L.g.b, g.data() + c * 5 * N, N, fn, a2, b2, t + 5 + 5 * c);
            t[20] = L.g.fJ[((size_t)en * 6 + fn) * NF + b2 * n1 + a2];
          }
        }
    }
}

// FR/CPR residual of one hexahedron, R = -div f (eq. eqn:FR_diff, d = 3):
// contravariant fluxes F^i = f . J a^i at the solution points, the Lagrange
// derivative along each reference direction, and the DG correction of the
// jumps between the common normal flux (Roe, through the outward J a^d of the
// face point) and the extrapolated flux polynomial.  Neighbours frozen.
//
// With mu > 0 the flux is f_inv - f_vis, with the two-dimensional scheme
// carried over direction by direction: at a solution point the viscous flux
// takes the corrected gradient (reference derivatives plus the DG correction
// of q_com - q^- on the two faces of each reference line, eq. com_q, then the
// chain rule); at a face point it takes q_com and the common gradient of eq.
// com_grad_q, the mean of both sides' broken gradients plus their BR2
// liftings eta_f g'(1) (q_com - q^(+-)) S^(+-) / |J|^(+-) (S the outward
// area-scaled normal, |J| the map's at the face point).  Boundary faces: the
// ghost side mirrors the own gradient and |J|; walls carry no viscous energy
// flux.
template <class S>
static void element_residual3(const Oracle3* o, const Level3& L, int e, const S* qe, const double* ntr, S* Re) {
  const Basis1D& b = L.g.b;
  const int P = L.g.P, n1 = L.g.n1, N = L.g.N, NF = L.g.NF;
  const Phys& ph = o->ph;
  const bool visc = ph.mu > 0.0;
  const double eta_f = 4.0, gface = 0.5 * n1 * n1;
  // own and other-side traces and the common state at every face point
  std::vector<S> qm_all(6 * NF * 5), qp_all(6 * NF * 5), qc_all(6 * NF * 5);
  for (int f = 0; f < 6; ++f) {
    const int en = o->nbr[(e * 6 + f) * 3], bc = o->nbr[(e * 6 + f) * 3 + 1];
    for (int fp = 0; fp < NF; ++fp) {
      const int a = fp % n1, bb = fp / n1;
      S* qm = &qm_all[(f * NF + fp) * 5];
      S* qp = &qp_all[(f * NF + fp) * 5];
      trace_state3(b, qe, N, f, a, bb, qm);
      const double* Sv = &L.g.fS[(((size_t)e * 6 + f) * NF + fp) * 3];
      if (en < 0) {
        double dS = std::sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
        double nu[3] = {Sv[0] / dS, Sv[1] / dS, Sv[2] / dS};
        ghost_state3(bc, qm, nu, o->cfg.q_inf, qp);
      } else {
        const double* t = &ntr[(((size_t)e * 6 + f) * NF + fp) * NT3];
        for (int v = 0; v < 5; ++v) qp[v] = t[v];
      }
      for (int v = 0; v < 5; ++v) qc_all[(f * NF + fp) * 5 + v] = 0.5 * (qm[v] + qp[v]);
    }
  }
  // corrected gradients at the solution points
  std::vector<S> gb, gc;
  if (visc) {
    gb.resize(15 * N);
    gc.resize(15 * N);
    broken_gradient3<S>(L, e, qe, gb.data());
    for (int v = 0; v < 5; ++v)
      for (int kk = 0; kk < n1; ++kk)
        for (int j = 0; j < n1; ++j)
          for (int i = 0; i < n1; ++i) {
            const int pt = (kk * n1 + j) * n1 + i, idx[3] = {i, j, kk};
            S dr[3] = {0.0, 0.0, 0.0};
            for (int m = 0; m < n1; ++m) {
              dr[0] += b.D[i * n1 + m] * qe[v * N + (kk * n1 + j) * n1 + m];
              dr[1] += b.D[j * n1 + m] * qe[v * N + (kk * n1 + m) * n1 + i];
              dr[2] += b.D[kk * n1 + m] * qe[v * N + (m * n1 + j) * n1 + i];
            }
            for (int d = 0; d < 3; ++d) {
              // face point of the line through pt on the faces 2d and 2d + 1
              const int a = d == 0 ? j : i, bb = d == 2 ? j : kk, fp = bb * n1 + a;
              const int fL = 2 * d, fR = 2 * d + 1;
              dr[d] += b.gL[idx[d]] * (qc_all[(fL * NF + fp) * 5 + v] - qm_all[(fL * NF + fp) * 5 + v]) +
                       b.gR[idx[d]] * (qc_all[(fR * NF + fp) * 5 + v] - qm_all[(fR * NF + fp) * 5 + v]);
            }
            const double* ja = &L.g.Ja[((size_t)e * N + pt) * 9];
            const double J = L.g.J[(size_t)e * N + pt];
            for (int c = 0; c < 3; ++c)
              gc[(c * 5 + v) * N + pt] = (ja[0 * 3 + c] * dr[0] + ja[1 * 3 + c] * dr[1] + ja[2 * 3 + c] * dr[2]) / J;
          }
  }
  std::vector<S> Ft(3 * 5 * N);   // [i][v][pt]
  for (int pt = 0; pt < N; ++pt) {
    S q[5];
    for (int v = 0; v < 5; ++v) q[v] = qe[v * N + pt];
    S fv[15];
    if (visc) {
      S d[15];
      for (int c = 0; c < 15; ++c) d[c] = gc[c * N + pt];
      viscous_flux3(q, d, ph, fv);
    }
    for (int i = 0; i < 3; ++i) {
      const double* ja = &L.g.Ja[((size_t)e * N + pt) * 9 + i * 3];
      S f[5];
      euler_flux3(q, ja, ph, f);
      if (visc)
        for (int v = 0; v < 5; ++v) f[v] -= ja[0] * fv[v] + ja[1] * fv[5 + v] + ja[2] * fv[10 + v];
      for (int v = 0; v < 5; ++v) Ft[(i * 5 + v) * N + pt] = f[v];
    }
  }
  std::vector<S> acc(5 * N, S(0.0));
  for (int v = 0; v < 5; ++v)
    for (int kk = 0; kk < n1; ++kk)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          S s = 0.0;
          for (int m = 0; m < n1; ++m) {
            s += b.D[i * n1 + m] * Ft[(0 * 5 + v) * N + (kk * n1 + j) * n1 + m];
            s += b.D[j * n1 + m] * Ft[(1 * 5 + v) * N + (kk * n1 + m) * n1 + i];
            s += b.D[kk * n1 + m] * Ft[(2 * 5 + v) * N + (m * n1 + j) * n1 + i];
          }
          acc[v * N + (kk * n1 + j) * n1 + i] = s;
        }
  for (int f = 0; f < 6; ++f) {
    const int en = o->nbr[(e * 6 + f) * 3], bc = o->nbr[(e * 6 + f) * 3 + 1];
    const bool bnd = en < 0;
    const int d = f / 2;
    const double sg = (f & 1) ? 1.0 : -1.0;
    const std::vector<double>& l = (f & 1) ? b.lp : b.lm;
    const std::vector<double>& gp = (f & 1) ? b.gR : b.gL;
    for (int bb = 0; bb < n1; ++bb)
      for (int a = 0; a < n1; ++a) {
        const int fp = bb * n1 + a;
        S fo[5];
        const S* qm = &qm_all[(f * NF + fp) * 5];
        const S* qp = &qp_all[(f * NF + fp) * 5];
        const double* Sv = &L.g.fS[(((size_t)e * 6 + f) * NF + fp) * 3];
        roe_flux3(qm, qp, Sv, ph, fo);
        if (visc) {
          const double* t = &ntr[(((size_t)e * 6 + f) * NF + fp) * NT3];
          const double Jm = L.g.fJ[((size_t)e * 6 + f) * NF + fp], Jp = bnd ? Jm : t[20];
          S gm[15], gpv[15], dcom[15], qcm[5], fv[15];
          for (int c = 0; c < 3; ++c) trace_state3(b, gb.data() + c * 5 * N, N, f, a, bb, gm + 5 * c);
          for (int c = 0; c < 15; ++c) gpv[c] = bnd ? gm[c] : S(t[5 + c]);
          for (int v = 0; v < 5; ++v) {
            const S qcv = qc_all[(f * NF + fp) * 5 + v];
            qcm[v] = qcv;
            const S rm = eta_f * gface * (qcv - qm[v]) / Jm;   // times S_out
            const S rp = eta_f * gface * (qcv - qp[v]) / Jp;   // times -S_out
            for (int c = 0; c < 3; ++c) dcom[c * 5 + v] = 0.5 * (gm[c * 5 + v] + gpv[c * 5 + v] + (rm - rp) * Sv[c]);
          }
          viscous_flux3(qcm, dcom, ph, fv);
          const int nv = (bnd && bc != 4) ? 4 : 5;   // walls: no viscous energy flux
          for (int v = 0; v < nv; ++v) fo[v] -= fv[v] * Sv[0] + fv[5 + v] * Sv[1] + fv[10 + v] * Sv[2];
        }
        for (int v = 0; v < 5; ++v) {
          S loc = 0.0;
          for (int m = 0; m < n1; ++m) loc += l[m] * Ft[(d * 5 + v) * N + line_pt3(P, f, a, bb, m)];
          S jump = sg * fo[v] - loc;
          for (int m = 0; m < n1; ++m) acc[v * N + line_pt3(P, f, a, bb, m)] += gp[m] * jump;
        }
      }
  }
  for (int v = 0; v < 5; ++v)
    for (int pt = 0; pt < N; ++pt) Re[v * N + pt] = -acc[v * N + pt] / L.g.J[(size_t)e * N + pt];
}

static void full_residual3(const Oracle3* o, const Level3& L, const double* q, double* R) {
  const int N = L.g.N, E = o->E;
  std::vector<double> tr;
  neighbour_traces3(o, L, q, tr);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int e = 0; e < E; ++e) {
    std::vector<double> qe(5 * N), Re(5 * N);
    for (int v = 0; v < 5; ++v)
      for (int p = 0; p < N; ++p) qe[v * N + p] = q[((size_t)v * E + e) * N + p];
    element_residual3<double>(o, L, e, qe.data(), tr.data(), Re.data());
    for (int v = 0; v < 5; ++v)
      for (int p = 0; p < N; ++p) R[((size_t)v * E + e) * N + p] = Re[v * N + p];
  }
}

// Level system F_l(q) - S_l, eq. ESDIRK_primitive (coarse levels without the
// stage source, which cancels against S_l: the 2D reading).
static void level_F3(const Oracle3* o, int l, const double* q, bool with_src, bool minus_S, double* F) {
  const Level3& L = o->lev[l];
  const int N = L.g.N, E = o->E;
  const size_t tot = (size_t)5 * E * N;
  full_residual3(o, L, q, F);
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qq[5], qc[5];
      for (int v = 0; v < 5; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
      cons_from_prim3(qq, o->ph, qc);
      for (int v = 0; v < 5; ++v) {
        size_t id = ((size_t)v * E + e) * N + p;
        F[id] += -qc[v] / o->omega_dt;
        if (with_src) F[id] += o->src[id];
      }
    }
  if (minus_S)
    for (size_t i = 0; i < tot; ++i) F[i] -= L.S[i];
}

// Element block D_e = Gamma/dtau + M/(omega dt) - dR_e/dq_e by complex step.
static void element_block3(const Oracle3* o, const Level3& L, int e, const double* q, const double* ntr,
                           double dtau, double* Dm) {
  const int N = L.g.N, n = 5 * N, E = o->E;
  const double h = 1e-30;
  std::vector<cplx> qe(n), Re(n);
  for (int col = 0; col < n; ++col) {
    for (int v = 0; v < 5; ++v)
      for (int p = 0; p < N; ++p) qe[v * N + p] = cplx(q[((size_t)v * E + e) * N + p], 0.0);
    qe[col] += cplx(0.0, h);
    element_residual3<cplx>(o, L, e, qe.data(), ntr, Re.data());
    for (int row = 0; row < n; ++row) Dm[(size_t)row * n + col] = -Re[row].imag() / h;
  }
  for (int p = 0; p < N; ++p) {
    double qq[5];
    for (int v = 0; v < 5; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
    double eps = precond_eps3(qq, o->ph);
    double G[5][5], M[5][5];
    Gamma_matrix3(qq, eps, o->ph, G);
    M_matrix3(qq, o->ph, M);
    for (int a = 0; a < 5; ++a)
      for (int c = 0; c < 5; ++c)
        Dm[(size_t)(a * N + p) * n + (c * N + p)] += G[a][c] / dtau + M[a][c] / o->omega_dt;
  }
}

static int refresh_level3(Oracle3* o, int l) {
  Level3& L = o->lev[l];
  const int N = L.g.N, n = 5 * N, E = o->E;
  std::vector<double> tr;
  neighbour_traces3(o, L, L.q.data(), tr);
  L.lu.assign((size_t)E * n * n, 0.0);
  L.piv.assign((size_t)E * n, 0);
  int singular = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 2) reduction(| : singular)
#endif
  for (int e = 0; e < E; ++e) {
    double* Dm = &L.lu[(size_t)e * n * n];
    element_block3(o, L, e, L.q.data(), tr.data(), o->dtau, Dm);
    if (!lu_factor(n, Dm, &L.piv[(size_t)e * n])) singular |= 1;
  }
  return singular ? -4 : 0;
}

// Element-Jacobi sweeps, eq. smoothing_element_jacobi.
static void smooth3(Oracle3* o, int l, int nsweep) {
  Level3& L = o->lev[l];
  const int N = L.g.N, n = 5 * N, E = o->E;
  L.F.resize((size_t)5 * E * N);
  for (int s = 0; s < nsweep; ++s) {
    level_F3(o, l, L.q.data(), l == 0, l > 0, L.F.data());
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int e = 0; e < E; ++e) {
      std::vector<double> x(n);
      for (int v = 0; v < 5; ++v)
        for (int p = 0; p < N; ++p) x[v * N + p] = L.F[((size_t)v * E + e) * N + p];
      lu_solve(n, &L.lu[(size_t)e * n * n], &L.piv[(size_t)e * n], x.data());
      for (int v = 0; v < 5; ++v)
        for (int p = 0; p < N; ++p) L.q[((size_t)v * E + e) * N + p] += x[v * N + p];
    }
  }
}

// out[v][e][(k,j,i)] = sum op[i][a] op[j][b] op[k][c] in[v][e][(c,b,a)].
static void apply_tensor3(const std::vector<double>& op, int nout, int nin, int E, const double* in,
                          double* out) {
  const int Nin = nin * nin * nin, Nout = nout * nout * nout;
  for (int v = 0; v < 5; ++v)
    for (int e = 0; e < E; ++e)
      for (int k = 0; k < nout; ++k)
        for (int j = 0; j < nout; ++j)
          for (int i = 0; i < nout; ++i) {
            double s = 0.0;
            for (int c = 0; c < nin; ++c)
              for (int bb = 0; bb < nin; ++bb)
                for (int a = 0; a < nin; ++a)
                  s += op[i * nin + a] * op[j * nin + bb] * op[k * nin + c] *
                       in[((size_t)v * E + e) * Nin + (c * nin + bb) * nin + a];
            out[((size_t)v * E + e) * Nout + (k * nout + j) * nout + i] = s;
          }
}

// FAS V-cycle (Section 3), the 2D steps on hexahedra.
static int vcycle_level3(Oracle3* o, int l, bool refresh) {
  Level3& L = o->lev[l];
  const int E = o->E;
  if (refresh) { int st = refresh_level3(o, l); if (st) return st; }
  smooth3(o, l, o->cfg.n_smooth[l]);
  if (l == o->cfg.n_levels - 1) return 0;
  Level3& C = o->lev[l + 1];
  const int Nf = L.g.N, Nc = C.g.N;
  std::vector<double> d((size_t)5 * E * Nf);
  level_F3(o, l, L.q.data(), l == 0, l > 0, d.data());
  for (auto& x : d) x = -x;
  C.q.resize((size_t)5 * E * Nc);
  apply_tensor3(o->Rm[l], C.g.n1, L.g.n1, E, L.q.data(), C.q.data());
  C.qb = C.q;
  std::vector<double> Pd((size_t)5 * E * Nc), Fc((size_t)5 * E * Nc);
  apply_tensor3(o->Rm[l], C.g.n1, L.g.n1, E, d.data(), Pd.data());
  level_F3(o, l + 1, C.q.data(), false, false, Fc.data());
  C.S.resize((size_t)5 * E * Nc);
  for (size_t i = 0; i < C.S.size(); ++i) C.S[i] = Fc[i] + Pd[i];
  int st = vcycle_level3(o, l + 1, refresh);
  if (st) return st;
  std::vector<double> corr((size_t)5 * E * Nc), pc((size_t)5 * E * Nf);
  for (size_t i = 0; i < corr.size(); ++i) corr[i] = C.q[i] - C.qb[i];
  apply_tensor3(o->Pm[l], L.g.n1, C.g.n1, E, corr.data(), pc.data());
  for (size_t i = 0; i < pc.size(); ++i) L.q[i] += pc[i];
  smooth3(o, l, o->cfg.n_smooth[l]);
  return 0;
}

// ||F|| of eq. ser with each equation divided by its reference scale.
static double residual_norm3(const Oracle3* o, const std::vector<double>& F) {
  const size_t plane = F.size() / 5;
  double s = 0.0;
  for (int v = 0; v < 5; ++v) {
    double sc = o->cfg.res_scale[v] > 0.0 ? o->cfg.res_scale[v] : 1.0;
    double t = 0.0;
    for (size_t i = 0; i < plane; ++i) t += F[v * plane + i] * F[v * plane + i];
    s += t / (sc * sc);
  }
  return std::sqrt(s);
}

extern "C" {

int orc3_gll(int n, double* x) {
  std::vector<double> g = gll_nodes(n);
  for (int i = 0; i <= n; ++i) x[i] = g[i];
  return 0;
}

int orc3_point_matrices(const double* q, double gamma, double Ma_inf, double kappa, int cutoff, double* M,
                        double* G, double* eps_out) {
  Phys ph = {gamma, Ma_inf, kappa, cutoff};
  double MM[5][5], GG[5][5];
  double e = precond_eps3(q, ph);
  M_matrix3(q, ph, MM);
  Gamma_matrix3(q, e, ph, GG);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) { M[i * 5 + j] = MM[i][j]; G[i * 5 + j] = GG[i][j]; }
  *eps_out = e;
  return 0;
}

int orc3_flux(const double* q, const double* n, double gamma, double* f, double* A) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  euler_flux3(q, n, ph, f);
  double AA[5][5];
  flux_jacobian3(q, n, ph, AA);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) A[i * 5 + j] = AA[i][j];
  return 0;
}

int orc3_roe(const double* qm, const double* qp, const double* Sv, double gamma, double Ma_inf, double kappa,
             int cutoff, double* out) {
  Phys ph = {gamma, Ma_inf, kappa, cutoff};
  roe_flux3(qm, qp, Sv, ph, out);
  return 0;
}

int orc3_cons_from_prim(const double* q, double gamma, double* qc) {
  Phys ph = {gamma, 0.0, 1.0, 0};
  cons_from_prim3(q, ph, qc);
  return 0;
}

void* orc3_create(const OrcConfig3* cfg, int E, int Ng, const double* nodes, const int* nbr) {
  Oracle3* o = new Oracle3();
  o->cfg = *cfg;
  o->ph.gamma = cfg->gamma; o->ph.Ma_inf = cfg->Ma_inf; o->ph.kappa = cfg->kappa; o->ph.cutoff = cfg->cutoff;
  o->ph.mu = cfg->mu; o->ph.Pr = cfg->Pr > 0.0 ? cfg->Pr : 0.72;
  o->E = E; o->Ng = Ng;
  const int nn = (Ng + 1) * (Ng + 1) * (Ng + 1);
  o->nodes.assign(nodes, nodes + (size_t)E * nn * 3);
  o->nbr.assign(nbr, nbr + (size_t)E * 18);
  for (int i = 0; i < E * 6; ++i) {
    const int en = nbr[i * 3], fn = nbr[i * 3 + 1], orient = nbr[i * 3 + 2];
    // as in 2D: slip walls for inviscid runs only, no-slip walls need the cut-off
    const bool ok = en >= 0 ? (en < E && fn >= 0 && fn < 6 && orient >= 0 && orient < 8)
                            : (en == -1 && fn >= 2 && fn <= 4 && !(fn == 2 && cfg->mu > 0) &&
                               !(fn == 3 && !(cfg->cutoff && cfg->kappa * cfg->Ma_inf > 0)));
    if (!ok) { delete o; return nullptr; }
  }
  o->lev.resize(cfg->n_levels);
  for (int l = 0; l < cfg->n_levels; ++l) {
    build_level_geom3(o, cfg->P[l], &o->lev[l].g);
    const size_t tot = (size_t)5 * E * o->lev[l].g.N;
    o->lev[l].q.assign(tot, 0.0);
    o->lev[l].S.assign(tot, 0.0);
  }
  for (int l = 0; l + 1 < cfg->n_levels; ++l) {
    o->Rm.push_back(make_restriction(o->lev[l].g.b, o->lev[l + 1].g.b));
    o->Pm.push_back(make_prolongation(o->lev[l].g.b, o->lev[l + 1].g.b));
  }
  o->src.assign((size_t)5 * E * o->lev[0].g.N, 0.0);
  o->omega_dt = 1.0;
  o->dtau = cfg->dtau_init;
  o->s = esdirk_tableau(cfg->esdirk_stages > 0 ? cfg->esdirk_stages : 4, o->A, o->b, o->c);
  return o;
}

void orc3_destroy(void* h) { delete (Oracle3*)h; }

// Metric terms of a level: Ja (E, N, 3, 3), J (E, N), face normals (E, 6, NF, 3), coordinates (E, N, 3).
int orc3_geometry(void* h, int level, double* Ja, double* J, double* fS, double* xyz) {
  const LevelGeom3& g = ((Oracle3*)h)->lev[level].g;
  if (Ja) memcpy(Ja, g.Ja.data(), g.Ja.size() * 8);
  if (J) memcpy(J, g.J.data(), g.J.size() * 8);
  if (fS) memcpy(fS, g.fS.data(), g.fS.size() * 8);
  if (xyz) memcpy(xyz, g.xyz.data(), g.xyz.size() * 8);
  return 0;
}

int orc3_residual(void* h, int level, const double* q, double* R) {
  Oracle3* o = (Oracle3*)h;
  full_residual3(o, o->lev[level], q, R);
  return 0;
}

int orc3_set_stage(void* h, const double* src, double omega_dt) {
  Oracle3* o = (Oracle3*)h;
  memcpy(o->src.data(), src, o->src.size() * 8);
  o->omega_dt = omega_dt;
  return 0;
}

int orc3_stage_F(void* h, int level, const double* q, double* F) {
  level_F3((Oracle3*)h, level, q, level == 0, false, F);
  return 0;
}

int orc3_blocks(void* h, int level, const double* q, double dtau, double* D) {
  Oracle3* o = (Oracle3*)h;
  const Level3& L = o->lev[level];
  const int n = 5 * L.g.N;
  std::vector<double> tr;
  neighbour_traces3(o, L, q, tr);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 2)
#endif
  for (int e = 0; e < o->E; ++e) element_block3(o, L, e, q, tr.data(), dtau, D + (size_t)e * n * n);
  return 0;
}

int orc3_restrict(void* h, int lf, const double* qf, double* qc) {
  Oracle3* o = (Oracle3*)h;
  apply_tensor3(o->Rm[lf], o->lev[lf + 1].g.n1, o->lev[lf].g.n1, o->E, qf, qc);
  return 0;
}

int orc3_prolong(void* h, int lf, const double* qc, double* qf) {
  Oracle3* o = (Oracle3*)h;
  apply_tensor3(o->Pm[lf], o->lev[lf].g.n1, o->lev[lf + 1].g.n1, o->E, qc, qf);
  return 0;
}

// One V-cycle on the finest-level state q (in/out) with the current stage data.
int orc3_vcycle(void* h, double* q, double dtau, int refresh) {
  Oracle3* o = (Oracle3*)h;
  Level3& L = o->lev[0];
  memcpy(L.q.data(), q, L.q.size() * 8);
  o->dtau = dtau;
  int st = vcycle_level3(o, 0, refresh != 0);
  memcpy(q, L.q.data(), L.q.size() * 8);
  return st;
}

// Pseudo-transient continuation of one stage (Section 2.4), as stage_solve.
int orc3_stage_solve(void* h, double* q, int* iters, double* drop) {
  Oracle3* o = (Oracle3*)h;
  std::vector<double> F(o->lev[0].q.size());
  double dtau = o->cfg.dtau_init, dtau_max = o->cfg.dtau_max, n0 = 0.0, prev = 0.0, built = 0.0;
  for (int m = 0;; ++m) {
    level_F3(o, 0, q, true, false, F.data());
    double nm = residual_norm3(o, F);
    if (m == 0) n0 = nm;
    if (nm <= o->cfg.tol * n0 || n0 == 0.0) { *iters = m; *drop = n0 > 0 ? nm / n0 : 0.0; return 0; }
    if (!std::isfinite(nm)) { *iters = m; *drop = nm; return -5; }
    if (m >= o->cfg.max_pseudo) { *iters = m; *drop = nm / n0; return -6; }
    if (m > 0) dtau = ser_next(dtau, prev, nm, dtau_max);
    bool refresh = refresh_due(m, o->cfg.refresh_every, built, dtau_max, o->cfg.refresh_always != 0);
    if (refresh) built = dtau;
    int st = orc3_vcycle(o, q, dtau, refresh);
    if (st) return st;
    prev = nm;
  }
}

// One ESDIRK physical step (eq. ESDIRK_ns), as orc_esdirk_step.
int orc3_esdirk_step(void* h, double* q, double dt, int* iters, double* drops) {
  Oracle3* o = (Oracle3*)h;
  Level3& L = o->lev[0];
  const int E = o->E, N = L.g.N, s = o->s;
  const size_t tot = (size_t)5 * E * N;
  std::vector<double> qcn(tot), qi(q, q + tot);
  std::vector<std::vector<double>> Rs(s, std::vector<double>(tot));
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qq[5], qc[5];
      for (int v = 0; v < 5; ++v) qq[v] = q[((size_t)v * E + e) * N + p];
      cons_from_prim3(qq, o->ph, qc);
      for (int v = 0; v < 5; ++v) qcn[((size_t)v * E + e) * N + p] = qc[v];
    }
  full_residual3(o, L, qi.data(), Rs[0].data());
  o->omega_dt = o->A[1][1] * dt;
  for (int i = 1; i < s; ++i) {
    for (size_t k = 0; k < tot; ++k) {
      double acc = qcn[k];
      for (int j = 0; j < i; ++j) acc += dt * o->A[i][j] * Rs[j][k];
      o->src[k] = acc / o->omega_dt;
    }
    int st = orc3_stage_solve(o, qi.data(), &iters[i - 1], &drops[i - 1]);
    if (st) return st;
    full_residual3(o, L, qi.data(), Rs[i].data());
  }
  for (int e = 0; e < E; ++e)
    for (int p = 0; p < N; ++p) {
      double qc[5], qq[5];
      for (int v = 0; v < 5; ++v) {
        size_t k = ((size_t)v * E + e) * N + p;
        double acc = qcn[k];
        for (int i = 0; i < s; ++i) acc += dt * o->b[i] * Rs[i][k];
        qc[v] = acc;
      }
      prim_from_cons3(qc, o->ph, qq);
      for (int v = 0; v < 5; ++v) q[((size_t)v * E + e) * N + p] = qq[v];
    }
  return 0;
}

}  // extern "C"
