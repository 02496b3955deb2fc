// host_tables3.cpp -- metrics and face tables of hexahedral meshes, built once
// on the host in FP64 and uploaded (Section 2.3 with d = 3).
//
// The metric terms J a^i_n = J d(xi^i)/dx_n are taken in the conservative
// curl form: J a^i_n = -(d_j W^n_k - d_k W^n_j), (i, j, k) cyclic, where
// W^n_k = X_l dX_m/dxi_k ((n, m, l) cyclic) is interpolated at the
// Gauss-Lobatto points of degree Pg = max(P, Ng, 1) and differentiated
// exactly.  Their divergence vanishes identically, the face normal (the
// outward J a^d of the same polynomial at a face point) involves only the
// face's own Gauss-Lobatto values, so both elements of a face agree, and with
// Pg >= Ng the interpolated map gradient is exact, so translated (periodic)
// copies of a face agree too.  For P >= Ng the metric terms are polynomials
// of degree <= P in every direction and uniform flow is exactly steady.
#include "pmg_internal.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace pmg {

// Gauss-Lobatto points of degree n: -1, the roots of L_n', +1.  Newton on L_n'
// with L_n'' from (1 - x^2) L_n'' = 2 x L_n' - n (n + 1) L_n.
static std::vector<double> lobatto_points(int n) {
  std::vector<double> x(n + 1);
  x[0] = -1.0;
  x[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    double t = -std::cos(M_PI * i / n);
    for (int it = 0; it < 60; ++it) {
      double a = 1.0, b = t;   // L_{k-1}, L_k
      for (int k = 2; k <= n; ++k) {
        double c = ((2 * k - 1) * t * b - (k - 1) * a) / k;
        a = b;
        b = c;
      }
      double dL = n * (t * b - a) / (t * t - 1.0);
      double d2 = (2.0 * t * dL - n * (n + 1.0) * b) / (1.0 - t * t);
      double step = dL / d2;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[i] = t;
  }
  return x;
}

// Values and derivatives of the Lagrange basis of nodes x at t.
static void lagrange_vd(const std::vector<double>& x, double t, std::vector<double>& l, std::vector<double>& dl) {
  const int n = (int)x.size();
  l.assign(n, 0.0);
  dl.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double v = 1.0, d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == k) continue;
      const double den = x[k] - x[m];
      d = d * (t - x[m]) / den + v / den;   // product rule, one factor at a time
      v *= (t - x[m]) / den;
    }
    l[k] = v;
    dl[k] = d;
  }
}

// Map of one hexahedron (Lagrange nodes of order Ng at equispaced reference
// positions) and its derivative at reference point r: X[n], dX[n][k].
static void hex_map(int Ng, const double* xn, const double r[3], double X[3], double dX[3][3]) {
  std::vector<double> g(Ng + 1);
  for (int a = 0; a <= Ng; ++a) g[a] = -1.0 + 2.0 * a / Ng;
  std::vector<double> l[3], dl[3];
  for (int d = 0; d < 3; ++d) lagrange_vd(g, r[d], l[d], dl[d]);
  for (int n = 0; n < 3; ++n) {
    X[n] = 0.0;
    for (int k = 0; k < 3; ++k) dX[n][k] = 0.0;
  }
  for (int c = 0; c <= Ng; ++c)
    for (int b = 0; b <= Ng; ++b)
      for (int a = 0; a <= Ng; ++a) {
        const double* P = xn + ((c * (Ng + 1) + b) * (Ng + 1) + a) * 3;
        const double v = l[0][a] * l[1][b] * l[2][c];
        const double d0 = dl[0][a] * l[1][b] * l[2][c], d1 = l[0][a] * dl[1][b] * l[2][c],
                     d2 = l[0][a] * l[1][b] * dl[2][c];
        for (int n = 0; n < 3; ++n) {
          X[n] += v * P[n];
          dX[n][0] += d0 * P[n];
          dX[n][1] += d1 * P[n];
          dX[n][2] += d2 * P[n];
        }
      }
}

// J a^i_n at r from the interpolant of W (Gauss-Lobatto nodes gl, W per
// node [n*3 + k]).
static void curl_form(const std::vector<double>& gl, const std::vector<double>& W, const double r[3],
                      double Ja[3][3]) {
  const int ng = (int)gl.size();
  std::vector<double> l[3], dl[3];
  for (int d = 0; d < 3; ++d) lagrange_vd(gl, r[d], l[d], dl[d]);
  double dW[3][3][3] = {};   // d_j W^n_k
  for (int c = 0; c < ng; ++c)
    for (int b = 0; b < ng; ++b)
      for (int a = 0; a < ng; ++a) {
        const double* w = &W[(size_t)((c * ng + b) * ng + a) * 9];
        const double g[3] = {dl[0][a] * l[1][b] * l[2][c], l[0][a] * dl[1][b] * l[2][c], l[0][a] * l[1][b] * dl[2][c]};
        for (int n = 0; n < 3; ++n)
          for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) dW[n][k][j] += g[j] * w[n * 3 + k];
      }
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    for (int n = 0; n < 3; ++n) Ja[i][n] = -(dW[n][k][j] - dW[n][j][k]);
  }
}

void build_faces3(MeshHost& m) {
  m.faces.clear();
  for (int e = 0; e < m.E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int* nb = &m.nbr[(size_t)(e * 6 + f) * 3];
      if (nb[0] < 0) {
        if (nb[1] != PMG_BC_SLIP_WALL && nb[1] != PMG_BC_NOSLIP_WALL && nb[1] != PMG_BC_FARFIELD)
          throw std::runtime_error("hexahedral boundary faces are slip walls (2), no-slip walls (3) or far field (4)");
        m.faces.push_back({e, f, -1, nb[1], 0});
        continue;
      }
      if (nb[0] >= m.E || nb[1] < 0 || nb[1] > 5 || nb[2] < 0 || nb[2] > 7)
        throw std::runtime_error("bad hexahedral neighbour entry");
      const int* back = &m.nbr[(size_t)(nb[0] * 6 + nb[1]) * 3];
      if (back[0] != e || back[1] != f) throw std::runtime_error("hexahedral face neighbours are not symmetric");
      if (e < nb[0] || (e == nb[0] && f < nb[1])) m.faces.push_back({e, f, nb[0], nb[1], nb[2]});
    }
}

void build_level_geometry3(const MeshHost& m, const Ref1D& r, LevelGeomHost& g) {
  const int P = r.P, n1 = P + 1, N = n1 * n1 * n1, NF = n1 * n1, E = m.E, Ng = m.Ng;
  const int nn = (Ng + 1) * (Ng + 1) * (Ng + 1);
  const int Pg = std::max(std::max(P, Ng), 1);
  const std::vector<double> gl = lobatto_points(Pg);
  const int ng = Pg + 1;
  const size_t plane = (size_t)E * N;
  g.met.assign(10 * plane, 0.0);
  g.xy.assign(plane * 3, 0.0);
  g.face.assign((size_t)E * 6 * NF * 4, 0.0);
  g.fJinv.assign((size_t)E * 6 * NF, 0.0);
  std::vector<double> W((size_t)ng * ng * ng * 9);
  for (int e = 0; e < E; ++e) {
    const double* xn = &m.nodes[(size_t)e * nn * 3];
    for (int c = 0; c < ng; ++c)
      for (int b = 0; b < ng; ++b)
        for (int a = 0; a < ng; ++a) {
          const double rr[3] = {gl[a], gl[b], gl[c]};
          double X[3], dX[3][3];
          hex_map(Ng, xn, rr, X, dX);
          double* w = &W[(size_t)((c * ng + b) * ng + a) * 9];
          for (int n = 0; n < 3; ++n) {
            const int mm = (n + 1) % 3, l = (n + 2) % 3;
            for (int k = 0; k < 3; ++k) w[n * 3 + k] = X[l] * dX[mm][k];
          }
        }
    for (int kk = 0; kk < n1; ++kk)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          const int pt = (kk * n1 + j) * n1 + i;
          const double rr[3] = {r.x[i], r.x[j], r.x[kk]};
          double X[3], dX[3][3], Ja[3][3];
          hex_map(Ng, xn, rr, X, dX);
          curl_form(gl, W, rr, Ja);
          const size_t gi = (size_t)e * N + pt;
          for (int ii = 0; ii < 3; ++ii)
            for (int n = 0; n < 3; ++n) g.met[(ii * 3 + n) * plane + gi] = Ja[ii][n];
          const double J = dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
                           dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
                           dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
          if (!(J > 0.0)) throw std::runtime_error("hexahedron with non-positive Jacobian");
          g.met[9 * plane + gi] = 1.0 / J;
          for (int n = 0; n < 3; ++n) g.xy[gi * 3 + n] = X[n];
        }
    for (int f = 0; f < 6; ++f) {
      const int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const double sg = (f & 1) ? 1.0 : -1.0;
      for (int b = 0; b < n1; ++b)
        for (int a = 0; a < n1; ++a) {
          double rr[3];
          rr[d] = sg;
          rr[t1] = r.x[a];
          rr[t2] = r.x[b];
          double Ja[3][3];
          curl_form(gl, W, rr, Ja);
          const double S[3] = {sg * Ja[d][0], sg * Ja[d][1], sg * Ja[d][2]};
          const double dS = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
          double* o = &g.face[(((size_t)e * 6 + f) * NF + b * n1 + a) * 4];
          o[0] = S[0] / dS;
          o[1] = S[1] / dS;
          o[2] = S[2] / dS;
          o[3] = dS;
          // 1/|J| of the map at the face point (the BR2 lifting's scale)
          double X[3], dX[3][3];
          hex_map(Ng, xn, rr, X, dX);
          const double J = dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
                           dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
                           dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
          if (!(J > 0.0)) throw std::runtime_error("hexahedron with non-positive Jacobian on a face");
          g.fJinv[((size_t)e * 6 + f) * NF + b * n1 + a] = 1.0 / J;
        }
    }
  }
}

}  // namespace pmg
