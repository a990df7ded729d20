"""Pins of the oracle's p-multigrid components (Sec. 4)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from oracle import assembly, geometry, pmg


def _grid_laplacian(n):
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n, n))
    I = sp.identity(n)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


def test_ilut_no_dropping_is_exact_lu():
    """tau = 0 and unlimited fill: ILUT is the exact LU factorisation."""
    d = assembly.Discretisation(3, 3, geometry.QuarterAnnulus())
    A = (d.M + 0.05 * d.K).tocsr()
    L, U = pmg.ilut(A, droptol=0.0, fill=1e9)
    LU = (sp.identity(A.shape[0]) + L) @ U
    np.testing.assert_allclose(LU.toarray(), A.toarray(), atol=1e-14 * abs(A).max())
    # one smoothing step with the exact factors solves the system
    hi, lo = assembly.problem(3, 3, geometry.QuarterAnnulus())
    P = pmg.PMG(hi, lo, 0.05, droptol=0.0, fill=1e9)
    b = np.random.default_rng(2).standard_normal(hi.N)
    x = P.smooth(b, np.zeros(hi.N))
    np.testing.assert_allclose(P.A @ x, b, atol=1e-12)


def test_ilut_row_limits_and_diagonal():
    hi, _ = assembly.problem(4, 6, geometry.UnitSquare())
    A = (hi.M + 0.01 * hi.K).tocsr()
    L, U = pmg.ilut(A, droptol=1e-12, fill=1.0)
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert L.indptr[i + 1] - L.indptr[i] <= np.sum(cols < i)
        ucols = U.indices[U.indptr[i]:U.indptr[i + 1]]
        assert i in ucols
        assert len(ucols) - 1 <= np.sum(cols > i)
        assert np.all(L.indices[L.indptr[i]:L.indptr[i + 1]] < i)


def test_ilut_banded_is_exact_lu():
    """A banded matrix has no LU fill outside its band, and for rows past the
    bandwidth the count limit ceil(fill*nnz) with fill = 1 keeps every entry:
    ILUT(0, 1) is then the exact LU factorisation (1D B-spline M + cK, p = 4)."""
    d = assembly.Discretisation(4, 9, geometry.UnitSquare())
    # 1D matrices: one row of the tensor grid (first interior row block)
    n = d.n
    from oracle import bspline
    k = bspline.open_uniform_knots(4, 9)
    x, w = np.polynomial.legendre.leggauss(5)
    M1 = np.zeros((d.nb, d.nb)); K1 = np.zeros((d.nb, d.nb))
    for (a, b) in bspline.elements(k):
        q = 0.5 * (b - a) * x + 0.5 * (a + b); wq = 0.5 * (b - a) * w
        B = bspline.basis(k, 4, q); D = bspline.basis_deriv(k, 4, q)
        M1 += (B * wq[:, None]).T @ B; K1 += (D * wq[:, None]).T @ D
    A = sp.csr_matrix((M1 + 0.02 * K1)[1:-1, 1:-1])
    L, U = pmg.ilut(A, droptol=0.0, fill=1.0)
    LU = ((sp.identity(n) + L) @ U).toarray()
    np.testing.assert_allclose(LU, A.toarray(), atol=1e-15)


def test_ilut_large_droptol_is_jacobi():
    """Dropping every off-diagonal entry leaves L = 0 and U = diag(A): the ILUT
    smoothing step becomes a Jacobi step x + D^{-1}(b - A x)."""
    A = (_grid_laplacian(5) * 1.0).tocsr()
    L, U = pmg.ilut(A, droptol=10.0, fill=1.0)
    assert L.nnz == 0
    np.testing.assert_array_equal(U.toarray(), np.diag(A.diagonal()))


def test_level_schedule_closed_forms():
    n = 7
    # 1D bidiagonal: level(i) = i
    L1 = sp.diags([np.ones(n - 1)], [-1], shape=(n, n)).tocsr()
    assert list(pmg.level_schedule(L1)) == list(range(n))
    # 2D 5-point lower part: level = ix + iy
    A = _grid_laplacian(n)
    lev = pmg.level_schedule(sp.tril(A, -1).tocsr())
    ix, iy = np.meshgrid(np.arange(n), np.arange(n))
    assert np.array_equal(lev, (ix + iy).ravel())


def test_gauss_seidel_matches_textbook_loop():
    rng = np.random.default_rng(3)
    A = (_grid_laplacian(5) + sp.random(25, 25, density=0.1, random_state=4)).tocsr()
    A = (A + sp.identity(25) * 10).tocsr()
    b = rng.standard_normal(25)
    x0 = rng.standard_normal(25)
    x = x0.copy()
    Ad = A.toarray()
    for i in range(25):
        x[i] = (b[i] - Ad[i, :i] @ x[:i] - Ad[i, i + 1:] @ x[i + 1:]) / Ad[i, i]
    np.testing.assert_allclose(pmg.gauss_seidel(A, b, x0), x, rtol=1e-13)


def test_bilinear_prolongation_exact_for_bilinears():
    """Knot insertion: nodal values of a bilinear function on the coarse mesh are
    mapped exactly to its nodal values on the fine mesh."""
    nc = 4
    P1 = pmg.prolongation_1d(nc)
    P2 = sp.kron(P1, P1)
    xc = np.arange(1, nc) / nc
    xf = np.arange(1, 2 * nc) / (2 * nc)
    f = lambda x, y: x * y * (1 - x) * 0 + x * y  # bilinear, nonzero in the interior
    Xc, Yc = np.meshgrid(xc, xc)
    Xf, Yf = np.meshgrid(xf, xf)
    # a function vanishing on the boundary: use hat-compatible x(1-x) only at nodes
    # (bilinear interpolation is exact for piecewise-bilinear interpolants)
    coarse = (np.minimum(Xc, 1 - Xc) * np.minimum(Yc, 1 - Yc)).ravel()
    fine = P2 @ coarse
    # the interpolant of a piecewise-bilinear function at midpoints is its average
    want = np.array([[np.interp(x, np.r_[0, xc, 1], np.r_[0, np.minimum(xc, 1 - xc), 0]) *
                      np.interp(y, np.r_[0, xc, 1], np.r_[0, np.minimum(xc, 1 - xc), 0])
                      for x in xf] for y in xf]).ravel()
    np.testing.assert_allclose(fine, want, atol=1e-15)


def test_galerkin_coarse_equals_rediscretisation_q1():
    """For Q1 on the unit square the Galerkin operator P^T A_h P equals the
    operator assembled on the coarse mesh (nested spaces, exact integration)."""
    fine = assembly.Discretisation(1, 8, geometry.UnitSquare())
    coarse = assembly.Discretisation(1, 4, geometry.UnitSquare())
    A = (fine.M + 0.3 * fine.K).tocsr()
    h = pmg.HMG(A, 8, coarsest_nel=4)
    np.testing.assert_allclose(h.A[1].toarray(), (coarse.M + 0.3 * coarse.K).toarray(), atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_pmg_converges_to_direct(p):
    hi, lo = assembly.problem(p, 16, geometry.UnitSquare())
    P = pmg.PMG(hi, lo, 1.0 / 64)
    b = np.random.default_rng(p).standard_normal(hi.N)
    xd = spsolve(P.A.tocsc(), b)
    x = np.zeros(hi.N)
    r = [np.linalg.norm(b)]
    for _ in range(6):
        x = P.vcycle(b, x)
        r.append(np.linalg.norm(b - P.A @ x))
    rho = (r[4] / r[0]) ** 0.25
    assert rho < 0.1, r
    x, cyc = P.solve(b, np.zeros(hi.N), tol=1e-12)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-9 * np.abs(xd).max())
    assert cyc <= 8


def test_pmg_annulus_converges():
    hi, lo = assembly.problem(3, 8, geometry.QuarterAnnulus())
    P = pmg.PMG(hi, lo, 1.0 / 32)
    b = np.random.default_rng(7).standard_normal(hi.N)
    x, cyc = P.solve(b, np.zeros(hi.N), tol=1e-12)
    assert np.linalg.norm(b - P.A @ x) <= 1e-12 * np.linalg.norm(b)
    assert cyc <= 10
