// Host-side setup of the IgA discretisation and the p-multigrid hierarchy.
// Everything here runs once per problem (or per MGRIT level) on the CPU, in
// FP64, and produces plain arrays that csrc/capi.cu uploads to the device.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace igm {

// Row-compressed sparse matrix (host, FP64), columns ascending within a row.
struct Csr {
  int rows = 0, cols = 0;
  std::vector<int> ptr, col;
  std::vector<double> val;
  int nnz() const { return (int)col.size(); }
};

// Matrix on an n x n tensor grid of unknowns (i = ix + n*iy) whose row i
// couples only to (ix+dx, iy+dy) with |dx|,|dy| <= w.  val[i*(2w+1)^2 +
// (dy+w)*(2w+1) + (dx+w)]; entries that fall outside the grid are stored as 0.
struct Stencil {
  int n = 0, w = 0;
  std::vector<double> val;
  int width() const { return 2 * w + 1; }
  Csr to_csr(bool drop_zeros) const;
};

// Geometry: identity on the unit square, or a B-spline map with open uniform
// knots (degrees gdeg, gn control points per direction, ctrl [gn1][gn0][2]).
struct Geometry {
  bool affine = true;
  int deg[2] = {0, 0}, nctrl[2] = {0, 0};
  std::vector<double> knots[2];
  std::vector<double> ctrl;
  // F(xi,eta) and J[a][b] = d x_a / d xi_b
  void eval(double xi, double eta, double* x, double J[2][2]) const;
};

// One B-spline order on one uniform mesh of nel x nel elements.
struct Discretisation {
  int p = 0, nel = 0, nq = 0;
  int nb = 0;      // univariate functions per direction (nel + p)
  int n = 0;       // interior unknowns per direction (nb - 2)
  int N = 0;       // n * n
  std::vector<double> knots;
  Stencil M, K;    // interior x interior, w = p
  std::vector<double> lumped;   // interior rows of the full-basis row sums of M
  std::vector<double> M1, K1;   // affine only: interior 1D matrices, band [n][2p+1]
};

// Univariate helpers (own implementations; see host_setup.cpp).
std::vector<double> open_uniform_knots(int p, int nel);
void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w);  // on [-1,1]
// Values and first derivatives of the p+1 functions nonzero on knot span s
// (knots[s] <= x < knots[s+1]): functions s-p .. s.
void basis_on_span(const std::vector<double>& knots, int p, int s, double x, double* N, double* dN);
// Index s of the knot span holding x (knots[s] <= x < knots[s+1]; the last
// non-empty span at the right end).
int find_span(const std::vector<double>& knots, int p, double x);

// Assemble order p on nel elements with nq Gauss points per direction.
std::string assemble(const Geometry& g, int p, int nel, int nq, Discretisation& d);

// Transfer matrix P_ij = int Phi_{i,hi.p} Phi_{j,lo.p}, interior x interior.
Csr transfer(const Geometry& g, const Discretisation& hi, const Discretisation& lo);

// Quadrature points (xi, eta, x, y) and weights*|detJ| over the whole mesh in
// element order (ey outer, ex inner), points eta outer, xi inner.
void quadrature_points(const Geometry& g, const Discretisation& d, std::vector<double>& pts,
                       std::vector<double>& wdet);
// b_i = sum_q wdet_q f_q Phi_i(q) over interior i.
void load_vector(const Geometry& g, const Discretisation& d, const double* fq, std::vector<double>& b);

// Dual-threshold ILUT in natural order (Saad's ILUT(tau, lfil) with
// lfil = ceil(fill * nnz of the row part)).  L strictly lower (unit diagonal
// implied), U upper including the diagonal.  Returns "" or an error text.
std::string ilut(const Csr& A, double droptol, double fill, Csr& L, Csr& U);

// Block-row (grid-row) data of a triangular factor on an n x n grid:
// off-block entries (other grid rows) as CSR, plus the dense inverse of every
// diagonal block, packed (lower: row i holds j = 0..i; upper: row i holds
// j = i..n-1).  For a unit lower factor the diagonal 1 is included in the
// inverse.
struct BlockTri {
  int n = 0;
  Csr off;                  // N x N, entries outside the row's own grid row
  std::vector<double> inv;  // n blocks of n(n+1)/2
};
std::string block_lower(const Csr& L, int n, BlockTri& out);  // L strictly lower, unit diag
std::string block_upper(const Csr& U, int n, BlockTri& out);  // U with diagonal

// Galerkin coarse operator P^T A P for the bilinear prolongation from an
// (nc x nc)-unknown grid (nel_c elements) to the (2 nel_c - 1)^2 grid.
Stencil galerkin_coarse(const Stencil& A);

// Dense inverse of an SPD matrix via Cholesky (row-major n x n).
std::string spd_inverse(const Stencil& A, std::vector<double>& inv);

}  // namespace igm
