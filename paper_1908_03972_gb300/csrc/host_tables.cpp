// host_tables.cpp -- reference-element operators and mesh metrics, built once
// on the host in FP64 and uploaded (Section 2.3, Section 3).
//
//  * Gauss-Legendre points by Newton iteration on L_{P+1}, weights from L'.
//  * Lagrange differentiation and trace vectors in barycentric form.
//  * DG correction (Radau) derivatives through the nodal-DG lift identity
//    g_R'(x_i) = l_i(1)/w_i, g_L'(x_i) = -l_i(-1)/w_i.
//  * Restriction = L2 projection by truncation of Legendre modes (the modal
//    coefficients come from Gauss quadrature, exact at these degrees);
//    prolongation = barycentric evaluation of the coarse interpolant.
//  * Metrics from the geometry map written in monomials, evaluated exactly at
//    each level's own solution and flux points.
#include "pmg_internal.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace pmg {

static void legendre_pair(int n, double x, double* Ln, double* dLn) {
  // L_n and L_n' from the three-term recurrence and
  // L_n' = n (x L_n - L_{n-1}) / (x^2 - 1) (x is never +-1 here).
  double a = 1.0, b = x;
  if (n == 0) { *Ln = 1.0; *dLn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  *Ln = b;
  *dLn = n * (x * b - a) / (x * x - 1.0);
}

static double legendre_val(int k, double x) {
  double L, dL;
  if (k == 0) return 1.0;
  legendre_pair(k, x, &L, &dL);
  return L;
}

static void barycentric_weights(const std::vector<double>& x, std::vector<double>& lam) {
  int n = (int)x.size();
  lam.assign(n, 1.0);
  for (int k = 0; k < n; ++k)
    for (int m = 0; m < n; ++m)
      if (m != k) lam[k] /= (x[k] - x[m]);
}

// l_k(t) for all k by the barycentric formula (t may coincide with a node).
static void lagrange_at(const std::vector<double>& x, const std::vector<double>& lam, double t,
                        std::vector<double>& out) {
  int n = (int)x.size();
  out.assign(n, 0.0);
  for (int k = 0; k < n; ++k)
    if (t == x[k]) { out[k] = 1.0; return; }
  double s = 0.0;
  for (int k = 0; k < n; ++k) { out[k] = lam[k] / (t - x[k]); s += out[k]; }
  for (int k = 0; k < n; ++k) out[k] /= s;
}

Ref1D make_ref1d(int P) {
  Ref1D r;
  r.P = P;
  int n = P + 1;
  r.x.resize(n);
  r.w.resize(n);
  for (int i = 0; i < n; ++i) {
    // Chebyshev nodes as starting guesses, ascending.
    double t = -std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * n));
    for (int it = 0; it < 60; ++it) {
      double L, dL;
      legendre_pair(n, t, &L, &dL);
      double step = L / dL;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    double L, dL;
    legendre_pair(n, t, &L, &dL);
    r.x[i] = t;
    r.w[i] = 2.0 / ((1.0 - t * t) * dL * dL);
  }
  std::vector<double> lam;
  barycentric_weights(r.x, lam);
  r.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      double v = (lam[k] / lam[i]) / (r.x[i] - r.x[k]);
      r.D[i * n + k] = v;
      diag -= v;
    }
    r.D[i * n + i] = diag;
  }
  lagrange_at(r.x, lam, -1.0, r.lm);
  lagrange_at(r.x, lam, 1.0, r.lp);
  r.gL.resize(n);
  r.gR.resize(n);
  for (int i = 0; i < n; ++i) {
    r.gR[i] = r.lp[i] / r.w[i];
    r.gL[i] = -r.lm[i] / r.w[i];
  }
  return r;
}

void make_transfer(const Ref1D& f, const Ref1D& c, std::vector<double>& R, std::vector<double>& I) {
  int nf = f.P + 1, nc = c.P + 1;
  R.assign(nc * nf, 0.0);
  for (int i = 0; i < nc; ++i)
    for (int q = 0; q < nf; ++q) {
      double s = 0.0;
      for (int k = 0; k <= c.P; ++k)
        s += legendre_val(k, c.x[i]) * 0.5 * (2 * k + 1) * f.w[q] * legendre_val(k, f.x[q]);
      R[i * nf + q] = s;
    }
  std::vector<double> lam, row;
  barycentric_weights(c.x, lam);
  I.assign(nf * nc, 0.0);
  for (int i = 0; i < nf; ++i) {
    lagrange_at(c.x, lam, f.x[i], row);
    for (int k = 0; k < nc; ++k) I[i * nc + k] = row[k];
  }
}

// Geometry map of order Ng on equispaced nodes written in monomials t^a:
// coefficient matrix C (row a = power, column = node) with
// sum_a C[a][node] t^a = phi_node(t).
static std::vector<double> geom_monomials(int Ng) {
  int n = Ng + 1;
  std::vector<double> V(n * n), C(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = -1.0 + 2.0 * i / Ng;
    double pw = 1.0;
    for (int a = 0; a < n; ++a) { V[i * n + a] = pw; pw *= t; }
  }
  // invert the Vandermonde matrix by Gauss-Jordan (n <= 5)
  std::vector<double> A(V), Inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) Inv[i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    for (int j = 0; j < n; ++j) { std::swap(A[k * n + j], A[p * n + j]); std::swap(Inv[k * n + j], Inv[p * n + j]); }
    double d = A[k * n + k];
    for (int j = 0; j < n; ++j) { A[k * n + j] /= d; Inv[k * n + j] /= d; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      double f = A[i * n + k];
      for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[k * n + j]; Inv[i * n + j] -= f * Inv[k * n + j]; }
    }
  }
  // V C = I  ->  C = V^-1; phi_node(t) = sum_a C[a][node] t^a
  for (int a = 0; a < n; ++a)
    for (int node = 0; node < n; ++node) C[a * n + node] = Inv[a * n + node];
  return C;
}

static void geom_basis(const std::vector<double>& C, int Ng, double t, double* phi, double* dphi) {
  int n = Ng + 1;
  for (int node = 0; node < n; ++node) {
    double v = 0.0, d = 0.0;
    for (int a = n - 1; a >= 0; --a) {
      d = d * t + v;
      v = v * t + C[a * n + node];
    }
    phi[node] = v;
    dphi[node] = d;
  }
}

static void map_jacobian(const std::vector<double>& C, int Ng, const double* xn, double xi, double eta,
                         double* x, double* y, double J[4]) {
  double px[8], dpx[8], py[8], dpy[8];
  geom_basis(C, Ng, xi, px, dpx);
  geom_basis(C, Ng, eta, py, dpy);
  double xx = 0, yy = 0, x_xi = 0, x_eta = 0, y_xi = 0, y_eta = 0;
  for (int b = 0; b <= Ng; ++b)
    for (int a = 0; a <= Ng; ++a) {
      const double* X = xn + (b * (Ng + 1) + a) * 2;
      double s = px[a] * py[b], sx = dpx[a] * py[b], se = px[a] * dpy[b];
      xx += s * X[0]; yy += s * X[1];
      x_xi += sx * X[0]; x_eta += se * X[0];
      y_xi += sx * X[1]; y_eta += se * X[1];
    }
  *x = xx; *y = yy;
  J[0] = x_xi; J[1] = x_eta; J[2] = y_xi; J[3] = y_eta;
}

void build_level_geometry(const MeshHost& m, const Ref1D& r, LevelGeomHost& g) {
  int P = r.P, n1 = P + 1, N = n1 * n1, E = m.E, Ng = m.Ng, nn = (Ng + 1) * (Ng + 1);
  std::vector<double> C = geom_monomials(Ng);
  g.met.assign((size_t)5 * E * N, 0.0);
  g.xy.assign((size_t)E * N * 2, 0.0);
  g.face.assign((size_t)E * 4 * n1 * 3, 0.0);
  g.fJinv.assign((size_t)E * 4 * n1, 0.0);
  for (int e = 0; e < E; ++e) {
    const double* xn = &m.nodes[(size_t)e * nn * 2];
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        double x, y, J[4];
        map_jacobian(C, Ng, xn, r.x[i], r.x[j], &x, &y, J);
        size_t pt = (size_t)e * N + j * n1 + i;
        double det = J[0] * J[3] - J[1] * J[2];
        if (!(det > 0.0)) throw std::runtime_error("non-positive element Jacobian");
        // contravariant flux coefficients: Ft = a f + b g, Gt = c f + d g
        g.met[0 * (size_t)E * N + pt] = J[3];    //  y_eta
        g.met[1 * (size_t)E * N + pt] = -J[1];   // -x_eta
        g.met[2 * (size_t)E * N + pt] = -J[2];   // -y_xi
        g.met[3 * (size_t)E * N + pt] = J[0];    //  x_xi
        g.met[4 * (size_t)E * N + pt] = 1.0 / det;
        g.xy[pt * 2 + 0] = x;
        g.xy[pt * 2 + 1] = y;
      }
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < n1; ++k) {
        double xi = (f == 1) ? 1.0 : (f == 3) ? -1.0 : r.x[k];
        double eta = (f == 2) ? 1.0 : (f == 0) ? -1.0 : r.x[k];
        double x, y, J[4];
        map_jacobian(C, Ng, xn, xi, eta, &x, &y, J);
        // outward area-scaled normal: +-(y_eta, -x_eta) on xi faces,
        // +-(-y_xi, x_xi) on eta faces
        double sx, sy;
        if (f == 1) { sx = J[3]; sy = -J[1]; }
        else if (f == 3) { sx = -J[3]; sy = J[1]; }
        else if (f == 2) { sx = -J[2]; sy = J[0]; }
        else { sx = J[2]; sy = -J[0]; }
        double dS = std::sqrt(sx * sx + sy * sy);
        double* o = &g.face[(((size_t)e * 4 + f) * n1 + k) * 3];
        o[0] = sx / dS; o[1] = sy / dS; o[2] = dS;
        double det = J[0] * J[3] - J[1] * J[2];
        if (!(det > 0.0)) throw std::runtime_error("non-positive element Jacobian on a face");
        g.fJinv[((size_t)e * 4 + f) * n1 + k] = 1.0 / det;
      }
  }
  // Both sides of a face must see the same normal flux: copy the owner's
  // normal, negated, to the neighbour's matching points.
  for (const FaceRec& fr : m.faces) {
    if (fr.eR < 0) continue;   // boundary faces have one side
    for (int k = 0; k < n1; ++k) {
      int kr = fr.rev ? P - k : k;
      const double* a = &g.face[(((size_t)fr.eL * 4 + fr.fL) * n1 + k) * 3];
      double* b = &g.face[(((size_t)fr.eR * 4 + fr.fR) * n1 + kr) * 3];
      b[0] = -a[0]; b[1] = -a[1]; b[2] = a[2];
    }
  }
}

// Element size of the CFL form (Section 2.4): twice the distance from the
// element's area centroid (8-point Gauss quadrature) to its nearest face, each
// face curve taken as the polyline through 65 equispaced reference points.
std::vector<double> element_sizes(const MeshHost& m) {
  const int Ng = m.Ng, nn = (Ng + 1) * (Ng + 1);
  std::vector<double> C = geom_monomials(Ng);
  Ref1D q8 = make_ref1d(7);
  std::vector<double> dx(m.E);
  for (int e = 0; e < m.E; ++e) {
    const double* xn = &m.nodes[(size_t)e * nn * 2];
    double A = 0.0, cx = 0.0, cy = 0.0;
    for (int j = 0; j < 8; ++j)
      for (int i = 0; i < 8; ++i) {
        double x, y, J[4];
        map_jacobian(C, Ng, xn, q8.x[i], q8.x[j], &x, &y, J);
        const double w = q8.w[i] * q8.w[j] * (J[0] * J[3] - J[1] * J[2]);
        A += w;
        cx += w * x;
        cy += w * y;
      }
    cx /= A;
    cy /= A;
    double best = 1e300;
    const int K = 64;
    for (int f = 0; f < 4; ++f) {
      double px = 0.0, py = 0.0;
      for (int k = 0; k <= K; ++k) {
        const double t = -1.0 + 2.0 * k / K;
        const double xi = (f == 1) ? 1.0 : (f == 3) ? -1.0 : t;
        const double eta = (f == 2) ? 1.0 : (f == 0) ? -1.0 : t;
        double x, y, J[4];
        map_jacobian(C, Ng, xn, xi, eta, &x, &y, J);
        if (k > 0) {
          const double ex = x - px, ey = y - py, L2 = ex * ex + ey * ey;
          double sgm = L2 > 0.0 ? ((cx - px) * ex + (cy - py) * ey) / L2 : 0.0;
          sgm = std::min(1.0, std::max(0.0, sgm));
          const double ddx = px + sgm * ex - cx, ddy = py + sgm * ey - cy;
          best = std::min(best, std::sqrt(ddx * ddx + ddy * ddy));
        }
        px = x;
        py = y;
      }
    }
    dx[e] = 2.0 * best;
  }
  return dx;
}

void build_faces(MeshHost& m) {
  m.faces.clear();
  for (int e = 0; e < m.E; ++e)
    for (int f = 0; f < 4; ++f) {
      int en = m.nbr[(e * 4 + f) * 3 + 0], fn = m.nbr[(e * 4 + f) * 3 + 1], rev = m.nbr[(e * 4 + f) * 3 + 2];
      if (en == -1) {   // boundary face: fn is the boundary type
        if (fn < PMG_BC_SLIP_WALL || fn > PMG_BC_FARFIELD) throw std::runtime_error("bad boundary type");
        m.faces.push_back(FaceRec{e, f, -1, fn, 0});
        continue;
      }
      if (en < 0 || en >= m.E || fn < 0 || fn > 3) throw std::runtime_error("bad neighbour table");
      const int* back = &m.nbr[(en * 4 + fn) * 3];
      if (back[0] != e || back[1] != f || back[2] != rev) throw std::runtime_error("neighbour table is not symmetric");
      if (e < en || (e == en && f < fn)) m.faces.push_back(FaceRec{e, f, en, fn, rev});
    }
}

}  // namespace pmg

namespace pmg {

// Tiles of the multi-sweep coarse-level smoother (k_tile.cu).  Every element
// belongs to the core of exactly one tile.  The cores come from recursive
// coordinate bisection of the element centroids (split the longer extent at
// the median until a part holds at most `core` elements), so they are compact
// on any mesh; the halo of a core is `depth` layers of face neighbours.
// Elements are listed core first, then halo layer by layer, so that the first
// layer_end[d] elements of a tile are its core and halo layers 1..d.  Sweep s
// of a launch of n sweeps updates the elements up to layer n - s, whose
// neighbours all lie within layer n - s + 1, so the core ends the launch with
// the values of n plain sweeps.
static void bisect(std::vector<int>& ids, size_t lo, size_t hi, const std::vector<double>& cx,
                   const std::vector<double>& cy, int core, std::vector<std::vector<int>>& out) {
  if (hi - lo <= (size_t)core) {
    out.emplace_back(ids.begin() + lo, ids.begin() + hi);
    return;
  }
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (size_t i = lo; i < hi; ++i) {
    x0 = std::min(x0, cx[ids[i]]); x1 = std::max(x1, cx[ids[i]]);
    y0 = std::min(y0, cy[ids[i]]); y1 = std::max(y1, cy[ids[i]]);
  }
  const std::vector<double>& key = (x1 - x0 >= y1 - y0) ? cx : cy;
  const size_t mid = lo + (hi - lo) / 2;
  std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi,
                   [&](int a, int b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
  bisect(ids, lo, mid, cx, cy, core, out);
  bisect(ids, mid, hi, cx, cy, core, out);
}

TileSet build_tiles(const MeshHost& m, int core, int depth) {
  const int E = m.E, nn = (m.Ng + 1) * (m.Ng + 1);
  TileSet ts;
  ts.depth = depth;
  std::vector<double> cx(E, 0.0), cy(E, 0.0);
  for (int e = 0; e < E; ++e) {
    for (int a = 0; a < nn; ++a) {
      cx[e] += m.nodes[((size_t)e * nn + a) * 2];
      cy[e] += m.nodes[((size_t)e * nn + a) * 2 + 1];
    }
    cx[e] /= nn;
    cy[e] /= nn;
  }
  std::vector<int> ids(E);
  for (int e = 0; e < E; ++e) ids[e] = e;
  std::vector<std::vector<int>> cores;
  bisect(ids, 0, ids.size(), cx, cy, core, cores);
  std::vector<int> mark(E, -1);
  ts.n_tiles = (int)cores.size();
  ts.off.push_back(0);
  for (int t = 0; t < ts.n_tiles; ++t) {
    std::vector<int> list = cores[t];
    std::sort(list.begin(), list.end());
    for (int e : list) mark[e] = t;
    std::vector<int> ends{(int)list.size()};
    size_t lo = 0;
    for (int d = 1; d <= depth; ++d) {
      const size_t hi = list.size();
      for (size_t h = lo; h < hi; ++h)
        for (int f = 0; f < 4; ++f) {
          const int en = m.nbr[(size_t)(list[h] * 4 + f) * 3];
          if (en >= 0 && mark[en] != t) {
            mark[en] = t;
            list.push_back(en);
          }
        }
      lo = hi;
      ends.push_back((int)list.size());
    }
    for (int i = 0; i < (int)list.size(); ++i)
      for (int f = 0; f < 4; ++f) {
        const int en = m.nbr[(size_t)(list[i] * 4 + f) * 3];
        int ls = -1;
        for (int j = 0; j < (int)list.size() && en >= 0; ++j)
          if (list[j] == en) { ls = j; break; }
        if (ls < 0 && en >= 0 && i < ends[depth > 0 ? depth - 1 : 0] && depth > 0)
          throw std::runtime_error("tile halo does not close");
        ts.lnbr.push_back(ls);
      }
    for (int e : list) ts.elems.push_back(e);
    for (int d = 0; d <= depth; ++d) ts.layer_end.push_back(ends[d]);
    ts.off.push_back((int)ts.elems.size());
    ts.max_elems = std::max(ts.max_elems, (int)list.size());
  }
  return ts;
}

}  // namespace pmg
