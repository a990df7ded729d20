// Host-side setup: B-spline basis, Gauss rule, geometry map, Gauss-quadrature
// assembly (Sec. 2), L2 transfer matrix and lumping (Sec. 4, Eq. (PM)), ILUT
// (Sec. 4 smoother), block-row triangular data and the p=1 h-hierarchy
// (Sec. 4, Fig. 5).  Compiled with -ffp-contract=off so that every product
// and sum is rounded separately (the ILUT's arithmetic order is part of its
// definition here).
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <queue>
#include <utility>

namespace igm {

// ---------------------------------------------------------------------------
// Univariate B-splines
// ---------------------------------------------------------------------------
std::vector<double> open_uniform_knots(int p, int nel) {
  std::vector<double> k;
  for (int i = 0; i <= p; ++i) k.push_back(0.0);
  for (int e = 1; e < nel; ++e) k.push_back((double)e / (double)nel);
  for (int i = 0; i <= p; ++i) k.push_back(1.0);
  return k;
}

// Gauss--Legendre nodes and weights on [-1,1]: Newton iteration on the
// Legendre polynomial P_n evaluated by its three-term recurrence.
void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w) {
  x.assign(nq, 0.0);
  w.assign(nq, 0.0);
  const double pi = 3.14159265358979323846;
  // P_n(z) and P_{n-1}(z) by (k) P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}
  auto legendre = [nq](double z, double& pn, double& pm) {
    pn = z;
    pm = 1.0;
    for (int k = 2; k <= nq; ++k) {
      double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
      pm = pn;
      pn = pk;
    }
  };
  for (int i = 0; i < (nq + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (nq + 0.5));
    double pn, pm, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(z, pn, pm);
      dp = nq * (z * pn - pm) / (z * z - 1.0);  // P_n'(z)
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(z, pn, pm);
    dp = nq * (z * pn - pm) / (z * z - 1.0);
    x[i] = -z;
    x[nq - 1 - i] = z;
    w[i] = w[nq - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (nq % 2 == 1) x[nq / 2] = 0.0;
}

// Cox--de Boor on one knot span: the functions of degree q nonzero on span s
// are s-q .. s.  vals[q][k] holds phi_{s-q+k, q}(x).
static void span_table(const std::vector<double>& t, int p, int s, double x,
                       std::vector<std::vector<double>>& vals) {
  vals.assign(p + 1, std::vector<double>());
  vals[0] = {1.0};
  for (int q = 1; q <= p; ++q) {
    vals[q].assign(q + 1, 0.0);
    for (int k = 0; k <= q; ++k) {
      int i = s - q + k;
      double v = 0.0;
      // left term uses phi_{i,q-1} = vals[q-1][k-1] (functions s-q+1..s at degree q-1)
      if (k - 1 >= 0) {
        double d = t[i + q] - t[i];
        if (d > 0.0) v += (x - t[i]) / d * vals[q - 1][k - 1];
      }
      if (k <= q - 1) {
        double d = t[i + q + 1] - t[i + 1];
        if (d > 0.0) v += (t[i + q + 1] - x) / d * vals[q - 1][k];
      }
      vals[q][k] = v;
    }
  }
}

void basis_on_span(const std::vector<double>& t, int p, int s, double x, double* N, double* dN) {
  std::vector<std::vector<double>> v;
  span_table(t, p, s, x, v);
  for (int k = 0; k <= p; ++k) N[k] = v[p][k];
  if (!dN) return;
  for (int k = 0; k <= p; ++k) {
    int i = s - p + k;
    double d = 0.0;
    if (p > 0) {
      if (k - 1 >= 0) {
        double den = t[i + p] - t[i];
        if (den > 0.0) d += p / den * v[p - 1][k - 1];
      }
      if (k <= p - 1) {
        double den = t[i + p + 1] - t[i + 1];
        if (den > 0.0) d -= p / den * v[p - 1][k];
      }
    }
    dN[k] = d;
  }
}

int find_span(const std::vector<double>& t, int p, double x) {
  int nb = (int)t.size() - p - 1;
  if (x >= t[nb]) return nb - 1;  // right end: last non-empty span
  int lo = p, hi = nb;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

void Geometry::eval(double xi, double eta, double* X, double J[2][2]) const {
  if (affine) {
    X[0] = xi; X[1] = eta;
    J[0][0] = 1.0; J[0][1] = 0.0; J[1][0] = 0.0; J[1][1] = 1.0;
    return;
  }
  const int p0 = deg[0], p1 = deg[1];
  const int s0 = find_span(knots[0], p0, xi), s1 = find_span(knots[1], p1, eta);
  std::vector<double> N0(p0 + 1), D0(p0 + 1), N1(p1 + 1), D1(p1 + 1);
  basis_on_span(knots[0], p0, s0, xi, N0.data(), D0.data());
  basis_on_span(knots[1], p1, s1, eta, N1.data(), D1.data());
  double x[2] = {0, 0}, dxi[2] = {0, 0}, deta[2] = {0, 0};
  for (int b = 0; b <= p1; ++b)
    for (int a = 0; a <= p0; ++a) {
      int ia = s0 - p0 + a, ib = s1 - p1 + b;
      const double* P = &ctrl[2 * (ia + nctrl[0] * ib)];
      for (int c = 0; c < 2; ++c) {
        x[c] += N0[a] * N1[b] * P[c];
        dxi[c] += D0[a] * N1[b] * P[c];
        deta[c] += N0[a] * D1[b] * P[c];
      }
    }
  X[0] = x[0]; X[1] = x[1];
  J[0][0] = dxi[0]; J[0][1] = deta[0];
  J[1][0] = dxi[1]; J[1][1] = deta[1];
}

// ---------------------------------------------------------------------------
// Assembly
// ---------------------------------------------------------------------------
Csr Stencil::to_csr(bool drop_zeros) const {
  Csr c;
  int N = n * n, W = width();
  c.rows = c.cols = N;
  c.ptr.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    int ix = i % n, iy = i / n;
    for (int dy = -w; dy <= w; ++dy)
      for (int dx = -w; dx <= w; ++dx) {
        int jx = ix + dx, jy = iy + dy;
        if (jx < 0 || jy < 0 || jx >= n || jy >= n) continue;
        double v = val[(size_t)i * W * W + (dy + w) * W + (dx + w)];
        if (drop_zeros && v == 0.0) continue;
        c.col.push_back(jx + n * jy);
        c.val.push_back(v);
      }
    c.ptr[i + 1] = (int)c.col.size();
  }
  return c;
}

struct ElemQuad {
  std::vector<double> xi, eta, wdet, X, Y;
  std::vector<double> JinvT;  // [q][2][2]
};

static void element_quadrature(const Geometry& g, const std::vector<double>& gx,
                               const std::vector<double>& gw, double x0, double x1, double y0,
                               double y1, ElemQuad& q, std::string* err) {
  int nq = (int)gx.size();
  q.xi.resize(nq * nq); q.eta.resize(nq * nq); q.wdet.resize(nq * nq);
  q.X.resize(nq * nq); q.Y.resize(nq * nq); q.JinvT.resize(4 * nq * nq);
  for (int b = 0; b < nq; ++b)
    for (int a = 0; a < nq; ++a) {
      int k = a + nq * b;
      double xi = 0.5 * (x1 - x0) * gx[a] + 0.5 * (x0 + x1);
      double eta = 0.5 * (y1 - y0) * gx[b] + 0.5 * (y0 + y1);
      double w = (0.5 * (x1 - x0) * gw[a]) * (0.5 * (y1 - y0) * gw[b]);
      double X[2], J[2][2];
      g.eval(xi, eta, X, J);
      double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      if (det == 0.0 && err) *err = "singular geometry Jacobian";
      q.xi[k] = xi; q.eta[k] = eta; q.X[k] = X[0]; q.Y[k] = X[1];
      q.wdet[k] = w * std::fabs(det);
      // J^{-T}: (J^{-1})^T = 1/det [[J11, -J10], [-J01, J00]]
      q.JinvT[4 * k + 0] = J[1][1] / det;
      q.JinvT[4 * k + 1] = -J[1][0] / det;
      q.JinvT[4 * k + 2] = -J[0][1] / det;
      q.JinvT[4 * k + 3] = J[0][0] / det;
    }
}

std::string assemble(const Geometry& g, int p, int nel, int nq, Discretisation& d) {
  if (p < 1 || nel < 2) return "need p >= 1 and nel >= 2";
  d.p = p; d.nel = nel; d.nq = nq;
  d.knots = open_uniform_knots(p, nel);
  d.nb = nel + p;
  d.n = d.nb - 2;
  d.N = d.n * d.n;
  if (d.n < 1) return "no interior unknowns";
  const int n = d.n, W = 2 * p + 1;
  d.M.n = d.K.n = n;
  d.M.w = d.K.w = p;
  d.M.val.assign((size_t)d.N * W * W, 0.0);
  d.K.val.assign((size_t)d.N * W * W, 0.0);
  std::vector<double> lumped_full((size_t)d.nb * d.nb, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  std::string err;
  std::vector<double> Nx((size_t)nq * (p + 1)), Dx((size_t)nq * (p + 1));
  std::vector<double> Ny((size_t)nq * (p + 1)), Dy((size_t)nq * (p + 1));
  ElemQuad q;
  const int nloc = (p + 1) * (p + 1);
  std::vector<double> V(nloc), G0(nloc), G1(nloc);
  for (int ey = 0; ey < nel; ++ey) {
    double y0 = d.knots[ey + p], y1 = d.knots[ey + p + 1];
    for (int ex = 0; ex < nel; ++ex) {
      double x0 = d.knots[ex + p], x1 = d.knots[ex + p + 1];
      element_quadrature(g, gx, gw, x0, x1, y0, y1, q, &err);
      if (!err.empty()) return err;
      for (int a = 0; a < nq; ++a) {
        basis_on_span(d.knots, p, ex + p, q.xi[a], &Nx[a * (p + 1)], &Dx[a * (p + 1)]);
        basis_on_span(d.knots, p, ey + p, q.eta[a * nq], &Ny[a * (p + 1)], &Dy[a * (p + 1)]);
      }
      for (int qb = 0; qb < nq; ++qb)
        for (int qa = 0; qa < nq; ++qa) {
          int k = qa + nq * qb;
          const double* JT = &q.JinvT[4 * k];
          for (int lb = 0; lb <= p; ++lb)
            for (int la = 0; la <= p; ++la) {
              int l = la + (p + 1) * lb;
              double vx = Nx[qa * (p + 1) + la], dvx = Dx[qa * (p + 1) + la];
              double vy = Ny[qb * (p + 1) + lb], dvy = Dy[qb * (p + 1) + lb];
              double gxi = dvx * vy, geta = vx * dvy;
              V[l] = vx * vy;
              G0[l] = JT[0] * gxi + JT[1] * geta;
              G1[l] = JT[2] * gxi + JT[3] * geta;
            }
          double wd = q.wdet[k];
          for (int la = 0; la < nloc; ++la) {
            int ax = ex + la % (p + 1), ay = ey + la / (p + 1);
            lumped_full[ax + (size_t)d.nb * ay] += wd * V[la];
            if (ax < 1 || ay < 1 || ax > d.nb - 2 || ay > d.nb - 2) continue;
            int row = (ax - 1) + n * (ay - 1);
            for (int lb = 0; lb < nloc; ++lb) {
              int bx = ex + lb % (p + 1), by = ey + lb / (p + 1);
              if (bx < 1 || by < 1 || bx > d.nb - 2 || by > d.nb - 2) continue;
              int dx = bx - ax, dy = by - ay;
              size_t idx = (size_t)row * W * W + (dy + p) * W + (dx + p);
              d.M.val[idx] += wd * V[la] * V[lb];
              d.K.val[idx] += wd * (G0[la] * G0[lb] + G1[la] * G1[lb]);
            }
          }
        }
    }
  }
  d.lumped.resize(d.N);
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix) d.lumped[ix + n * iy] = lumped_full[(ix + 1) + (size_t)d.nb * (iy + 1)];
  // 1D interior matrices for sum factorisation on the affine map
  if (g.affine) {
    d.M1.assign((size_t)n * W, 0.0);
    d.K1.assign((size_t)n * W, 0.0);
    std::vector<double> N1(p + 1), D1(p + 1);
    for (int e = 0; e < nel; ++e) {
      double x0 = d.knots[e + p], x1 = d.knots[e + p + 1];
      for (int a = 0; a < nq; ++a) {
        double x = 0.5 * (x1 - x0) * gx[a] + 0.5 * (x0 + x1);
        double w = 0.5 * (x1 - x0) * gw[a];
        basis_on_span(d.knots, p, e + p, x, N1.data(), D1.data());
        for (int la = 0; la <= p; ++la)
          for (int lb = 0; lb <= p; ++lb) {
            int ia = e + la, ib = e + lb;
            if (ia < 1 || ib < 1 || ia > d.nb - 2 || ib > d.nb - 2) continue;
            int row = ia - 1, off = ib - ia + p;
            d.M1[(size_t)row * W + off] += w * N1[la] * N1[lb];
            d.K1[(size_t)row * W + off] += w * D1[la] * D1[lb];
          }
      }
    }
  }
  return "";
}

Csr transfer(const Geometry& g, const Discretisation& hi, const Discretisation& lo) {
  // P_ij = int Phi_{i,hi} Phi_{j,lo} over interior i, j (same mesh, hi's rule)
  const int p = hi.p, pl = lo.p, nel = hi.nel, nq = hi.nq;
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  // accumulate into a per-row map: row i has columns within a (p+2) x (p+2) window
  int wx = p + pl + 1;  // window width in lo indices
  std::vector<double> acc((size_t)hi.N * wx * wx, 0.0);
  ElemQuad q;
  std::vector<double> Nx(p + 1), Ny(p + 1), Lx(pl + 1), Ly(pl + 1);
  for (int ey = 0; ey < nel; ++ey)
    for (int ex = 0; ex < nel; ++ex) {
      double x0 = hi.knots[ex + p], x1 = hi.knots[ex + p + 1];
      double y0 = hi.knots[ey + p], y1 = hi.knots[ey + p + 1];
      element_quadrature(g, gx, gw, x0, x1, y0, y1, q, nullptr);
      for (int qb = 0; qb < nq; ++qb)
        for (int qa = 0; qa < nq; ++qa) {
          int k = qa + nq * qb;
          basis_on_span(hi.knots, p, ex + p, q.xi[k], Nx.data(), nullptr);
          basis_on_span(hi.knots, p, ey + p, q.eta[k], Ny.data(), nullptr);
          basis_on_span(lo.knots, pl, ex + pl, q.xi[k], Lx.data(), nullptr);
          basis_on_span(lo.knots, pl, ey + pl, q.eta[k], Ly.data(), nullptr);
          for (int hb = 0; hb <= p; ++hb)
            for (int ha = 0; ha <= p; ++ha) {
              int ax = ex + ha, ay = ey + hb;
              if (ax < 1 || ay < 1 || ax > hi.nb - 2 || ay > hi.nb - 2) continue;
              int row = (ax - 1) + hi.n * (ay - 1);
              double vh = Nx[ha] * Ny[hb] * q.wdet[k];
              for (int lb = 0; lb <= pl; ++lb)
                for (int la = 0; la <= pl; ++la) {
                  int bx = ex + la, by = ey + lb;
                  if (bx < 1 || by < 1 || bx > lo.nb - 2 || by > lo.nb - 2) continue;
                  // window origin for row (ax, ay): lo index ax - p .. ax + pl
                  int ox = bx - (ax - p), oy = by - (ay - p);
                  acc[(size_t)row * wx * wx + oy * wx + ox] += vh * Lx[la] * Ly[lb];
                }
            }
        }
    }
  Csr P;
  P.rows = hi.N;
  P.cols = lo.N;
  P.ptr.assign(hi.N + 1, 0);
  for (int i = 0; i < hi.N; ++i) {
    int ax = i % hi.n + 1, ay = i / hi.n + 1;
    for (int oy = 0; oy < wx; ++oy)
      for (int ox = 0; ox < wx; ++ox) {
        int bx = ax - p + ox, by = ay - p + oy;
        if (bx < 1 || by < 1 || bx > lo.nb - 2 || by > lo.nb - 2) continue;
        double v = acc[(size_t)i * wx * wx + oy * wx + ox];
        if (v == 0.0) continue;
        P.col.push_back((bx - 1) + lo.n * (by - 1));
        P.val.push_back(v);
      }
    P.ptr[i + 1] = (int)P.col.size();
  }
  return P;
}

void quadrature_points(const Geometry& g, const Discretisation& d, std::vector<double>& pts,
                       std::vector<double>& wdet) {
  std::vector<double> gx, gw;
  gauss_legendre(d.nq, gx, gw);
  pts.clear();
  wdet.clear();
  ElemQuad q;
  for (int ey = 0; ey < d.nel; ++ey)
    for (int ex = 0; ex < d.nel; ++ex) {
      element_quadrature(g, gx, gw, d.knots[ex + d.p], d.knots[ex + d.p + 1], d.knots[ey + d.p],
                         d.knots[ey + d.p + 1], q, nullptr);
      for (size_t k = 0; k < q.xi.size(); ++k) {
        pts.push_back(q.xi[k]); pts.push_back(q.eta[k]);
        pts.push_back(q.X[k]); pts.push_back(q.Y[k]);
        wdet.push_back(q.wdet[k]);
      }
    }
}

void load_vector(const Geometry& g, const Discretisation& d, const double* fq, std::vector<double>& b) {
  std::vector<double> pts, wdet;
  quadrature_points(g, d, pts, wdet);
  const int p = d.p, nq = d.nq;
  b.assign(d.N, 0.0);
  std::vector<double> Nx(p + 1), Ny(p + 1);
  size_t k = 0;
  for (int ey = 0; ey < d.nel; ++ey)
    for (int ex = 0; ex < d.nel; ++ex)
      for (int qq = 0; qq < nq * nq; ++qq, ++k) {
        basis_on_span(d.knots, p, ex + p, pts[4 * k], Nx.data(), nullptr);
        basis_on_span(d.knots, p, ey + p, pts[4 * k + 1], Ny.data(), nullptr);
        double wf = wdet[k] * fq[k];
        for (int lb = 0; lb <= p; ++lb)
          for (int la = 0; la <= p; ++la) {
            int ax = ex + la, ay = ey + lb;
            if (ax < 1 || ay < 1 || ax > d.nb - 2 || ay > d.nb - 2) continue;
            b[(ax - 1) + d.n * (ay - 1)] += wf * Nx[la] * Ny[lb];
          }
      }
}

// ---------------------------------------------------------------------------
// ILUT (dual threshold, natural order)
// ---------------------------------------------------------------------------
std::string ilut(const Csr& A, double droptol, double fill, Csr& L, Csr& U) {
  const int n = A.rows;
  std::vector<double> w(n, 0.0);
  std::vector<char> inw(n, 0), seen(n, 0);
  std::vector<int> touched;
  std::vector<double> udiag(n, 0.0);
  // strictly-upper U rows kept for elimination of later rows
  std::vector<int> uptr(1, 0), ucol;
  std::vector<double> uval;
  L.rows = L.cols = U.rows = U.cols = n;
  L.ptr.assign(1, 0); L.col.clear(); L.val.clear();
  U.ptr.assign(1, 0); U.col.clear(); U.val.clear();
  std::vector<std::pair<int, double>> lower, upper;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    int nl = 0, nu = 0;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      double v = A.val[k];
      s += v * v;
      if (A.col[k] < i) ++nl;
      if (A.col[k] > i) ++nu;
    }
    const double tau = droptol * std::sqrt(s);
    const int lfil_l = (int)std::ceil(fill * nl), lfil_u = (int)std::ceil(fill * nu);
    std::priority_queue<int, std::vector<int>, std::greater<int>> heap;
    touched.clear();
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int c = A.col[k];
      w[c] = A.val[k];
      inw[c] = 1;
      touched.push_back(c);
      if (c < i) { heap.push(c); seen[c] = 1; }
    }
    while (!heap.empty()) {
      int k = heap.top();
      heap.pop();
      double wk = w[k] / udiag[k];
      if (std::fabs(wk) < tau) {
        inw[k] = 0;
        w[k] = 0.0;
        continue;
      }
      w[k] = wk;
      for (int e = uptr[k]; e < uptr[k + 1]; ++e) {
        int j = ucol[e];
        double ukj = uval[e];
        if (inw[j]) {
          w[j] = w[j] - wk * ukj;
        } else {
          w[j] = 0.0 - wk * ukj;
          inw[j] = 1;
          touched.push_back(j);
          if (j < i && !seen[j]) { heap.push(j); seen[j] = 1; }
        }
      }
    }
    if (!inw[i] || w[i] == 0.0) return "ILUT: zero pivot in row " + std::to_string(i);
    const double diag = w[i];
    lower.clear();
    upper.clear();
    for (int c : touched) {
      if (!inw[c]) continue;
      if (c < i && std::fabs(w[c]) >= tau) lower.emplace_back(c, w[c]);
      if (c > i && std::fabs(w[c]) >= tau) upper.emplace_back(c, w[c]);
    }
    auto bigger = [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
      double fa = std::fabs(a.second), fb = std::fabs(b.second);
      if (fa != fb) return fa > fb;
      return a.first < b.first;
    };
    std::sort(lower.begin(), lower.end(), bigger);
    std::sort(upper.begin(), upper.end(), bigger);
    if ((int)lower.size() > lfil_l) lower.resize(lfil_l);
    if ((int)upper.size() > lfil_u) upper.resize(lfil_u);
    std::sort(lower.begin(), lower.end());
    std::sort(upper.begin(), upper.end());
    for (auto& e : lower) { L.col.push_back(e.first); L.val.push_back(e.second); }
    L.ptr.push_back((int)L.col.size());
    U.col.push_back(i); U.val.push_back(diag);
    for (auto& e : upper) {
      U.col.push_back(e.first); U.val.push_back(e.second);
      ucol.push_back(e.first); uval.push_back(e.second);
    }
    U.ptr.push_back((int)U.col.size());
    uptr.push_back((int)ucol.size());
    udiag[i] = diag;
    for (int c : touched) { w[c] = 0.0; inw[c] = 0; seen[c] = 0; }
  }
  return "";
}

// ---------------------------------------------------------------------------
// Block-row data of triangular factors and Gauss--Seidel
// ---------------------------------------------------------------------------
static size_t lower_off(int i) { return (size_t)i * (i + 1) / 2; }
static size_t upper_off(int i, int n) { return (size_t)i * n - (size_t)i * (i - 1) / 2; }

std::string block_lower(const Csr& L, int n, BlockTri& out) {
  const int N = L.rows;
  if (N != n * n) return "block_lower: size mismatch";
  out.n = n;
  out.off.rows = out.off.cols = N;
  out.off.ptr.assign(1, 0); out.off.col.clear(); out.off.val.clear();
  out.inv.assign((size_t)n * lower_off(n), 0.0);
  std::vector<double> D((size_t)n * n);
  for (int by = 0; by < n; ++by) {
    std::fill(D.begin(), D.end(), 0.0);
    for (int r = 0; r < n; ++r) {
      int i = by * n + r;
      D[(size_t)r * n + r] = 1.0;
      for (int k = L.ptr[i]; k < L.ptr[i + 1]; ++k) {
        int c = L.col[k];
        if (c / n == by) D[(size_t)r * n + (c - by * n)] = L.val[k];
        else { out.off.col.push_back(c); out.off.val.push_back(L.val[k]); }
      }
      out.off.ptr.push_back((int)out.off.col.size());
    }
    // X = D^{-1}, column by column forward substitution
    double* inv = &out.inv[(size_t)by * lower_off(n)];
    std::vector<double> x(n);
    for (int j = 0; j < n; ++j) {
      for (int r = 0; r < n; ++r) x[r] = 0.0;
      x[j] = 1.0;
      for (int r = j + 1; r < n; ++r) {
        double s = 0.0;
        for (int l = j; l < r; ++l) s += D[(size_t)r * n + l] * x[l];
        x[r] = -s;
      }
      for (int r = j; r < n; ++r) inv[lower_off(r) + j] = x[r];
    }
  }
  return "";
}

std::string block_upper(const Csr& U, int n, BlockTri& out) {
  const int N = U.rows;
  if (N != n * n) return "block_upper: size mismatch";
  out.n = n;
  out.off.rows = out.off.cols = N;
  out.off.ptr.assign(1, 0); out.off.col.clear(); out.off.val.clear();
  out.inv.assign((size_t)n * upper_off(n, n), 0.0);
  std::vector<double> D((size_t)n * n);
  for (int by = 0; by < n; ++by) {
    std::fill(D.begin(), D.end(), 0.0);
    for (int r = 0; r < n; ++r) {
      int i = by * n + r;
      for (int k = U.ptr[i]; k < U.ptr[i + 1]; ++k) {
        int c = U.col[k];
        if (c / n == by) D[(size_t)r * n + (c - by * n)] = U.val[k];
        else { out.off.col.push_back(c); out.off.val.push_back(U.val[k]); }
      }
      out.off.ptr.push_back((int)out.off.col.size());
      if (D[(size_t)r * n + r] == 0.0) return "block_upper: zero diagonal";
    }
    double* inv = &out.inv[(size_t)by * upper_off(n, n)];
    std::vector<double> x(n);
    for (int j = 0; j < n; ++j) {
      for (int r = 0; r < n; ++r) x[r] = 0.0;
      x[j] = 1.0 / D[(size_t)j * n + j];
      for (int r = j - 1; r >= 0; --r) {
        double s = 0.0;
        for (int l = r + 1; l <= j; ++l) s += D[(size_t)r * n + l] * x[l];
        x[r] = -s / D[(size_t)r * n + r];
      }
      for (int r = 0; r <= j; ++r) inv[upper_off(r, n) + (j - r)] = x[r];
    }
  }
  return "";
}

Stencil galerkin_coarse(const Stencil& A) {
  // fine grid nf = 2 nc + 1 interior nodes per direction; coarse node J
  // (0-based c) sits at fine index 2c+1 with weights 1/2, 1, 1/2 on 2c, 2c+1, 2c+2.
  const int nf = A.n, nc = (nf - 1) / 2;
  Stencil C;
  C.n = nc;
  C.w = 1;
  C.val.assign((size_t)nc * nc * 9, 0.0);
  auto wt = [](int f, int c) -> double {  // 1D prolongation weight P[f][c]
    int d = f - (2 * c + 1);
    if (d == 0) return 1.0;
    if (d == 1 || d == -1) return 0.5;
    return 0.0;
  };
  for (int cy = 0; cy < nc; ++cy)
    for (int cx = 0; cx < nc; ++cx) {
      int I = cx + nc * cy;
      // sum over fine i in support of coarse I, fine j in stencil of i, coarse J near I
      for (int fy = 2 * cy; fy <= 2 * cy + 2; ++fy)
        for (int fx = 2 * cx; fx <= 2 * cx + 2; ++fx) {
          double pi = wt(fx, cx) * wt(fy, cy);
          if (pi == 0.0) continue;
          const double* a = &A.val[(size_t)(fx + nf * fy) * 9];
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int gx = fx + dx, gy = fy + dy;
              if (gx < 0 || gy < 0 || gx >= nf || gy >= nf) continue;
              double av = a[(dy + 1) * 3 + (dx + 1)];
              if (av == 0.0) continue;
              for (int ey = -1; ey <= 1; ++ey)
                for (int ex = -1; ex <= 1; ++ex) {
                  int jx = cx + ex, jy = cy + ey;
                  if (jx < 0 || jy < 0 || jx >= nc || jy >= nc) continue;
                  double pj = wt(gx, jx) * wt(gy, jy);
                  if (pj == 0.0) continue;
                  C.val[(size_t)I * 9 + (ey + 1) * 3 + (ex + 1)] += pi * av * pj;
                }
            }
        }
    }
  return C;
}

std::string spd_inverse(const Stencil& A, std::vector<double>& inv) {
  Csr c = A.to_csr(false);
  const int n = c.rows;
  std::vector<double> D((size_t)n * n, 0.0), Lc((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = c.ptr[i]; k < c.ptr[i + 1]; ++k) D[(size_t)i * n + c.col[k]] = c.val[k];
  for (int j = 0; j < n; ++j) {
    double s = D[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
    if (s <= 0.0) return "coarsest operator is not positive definite";
    double ljj = std::sqrt(s);
    Lc[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = D[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
      Lc[(size_t)i * n + j] = t / ljj;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> y(n), x(n);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= Lc[(size_t)i * n + k] * y[k];
      y[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= Lc[(size_t)k * n + i] * x[k];
      x[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + col] = x[i];
  }
  return "";
}

}  // namespace igm
