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


def _bilinear_prolongation_dense(nel_coarse):
    """Interior p = 1 nodes of nel_coarse elements -> interior nodes of
    2 nel_coarse elements, by linear interpolation written out from the nodal
    positions (x_c = c / nel_coarse, x_f = f / (2 nel_coarse)); tensor product
    in 2D with index ix + n iy."""
    nc, nf = nel_coarse - 1, 2 * nel_coarse - 1
    P1 = np.zeros((nf, nc))
    for f in range(1, nf + 1):            # fine node f at x = f / (2 nel_coarse)
        for c in range(1, nc + 1):        # coarse hat centred at x = 2c / (2 nel_coarse)
            d = abs(f - 2 * c)
            P1[f - 1, c - 1] = max(0.0, 1.0 - d / 2.0)
    return np.kron(P1, P1)


def test_hmg_cycle_is_a_w_cycle_gamma_2():
    """Fig. 5 (Sec. 4): one W-cycle visits each coarser level twice per visit of
    the level above.  On a three-level p = 1 hierarchy (32 -> 16 -> 8 elements)
    the cycle's error propagation operator is composed by hand from dense
    matrices: Gauss--Seidel S = I - (D + L)^{-1} A, Galerkin coarse operators
    P^T A P with the interpolation written out above, the exact solve on the
    coarsest level, and gamma = 2 coarse visits:
        E_k = S_k (I - P_k (I - E_{k+1}^2) A_{k+1}^{-1} P_k^T A_k) S_k,  E_last = 0.
    The oracle's cycle applied to x = e_j with b = 0 must reproduce column j.
    A V-cycle (gamma = 1), a missing smoothing step or a transposed transfer
    gives a different operator."""
    fine = assembly.Discretisation(1, 32, geometry.UnitSquare())
    A0 = (fine.M + 0.02 * fine.K).toarray()
    P01 = _bilinear_prolongation_dense(16)
    A1 = P01.T @ A0 @ P01
    P12 = _bilinear_prolongation_dense(8)
    A2 = P12.T @ A1 @ P12

    def smoother(A):
        return np.eye(A.shape[0]) - np.linalg.solve(np.tril(A), A)

    def two_grid(A, P, Ac, Ec):
        I = np.eye(A.shape[0])
        Ic = np.eye(Ac.shape[0])
        S = smoother(A)
        return S @ (I - P @ (Ic - Ec @ Ec) @ np.linalg.solve(Ac, P.T @ A)) @ S

    E2 = np.zeros_like(A2)
    E1 = two_grid(A1, P12, A2, E2)
    E0 = two_grid(A0, P01, A1, E1)
    h = pmg.HMG(sp.csr_matrix(A0), 32, coarsest_nel=8)
    assert len(h.A) == 3
    cols = np.stack([h.cycle(0, np.zeros(A0.shape[0]), e) for e in np.eye(A0.shape[0])], axis=1)
    np.testing.assert_allclose(cols, E0, atol=1e-12)
    # the V-cycle operator differs from it by far more than rounding
    E1v = two_grid(A1, P12, A2, E2)
    I1 = np.eye(A1.shape[0])
    S0 = smoother(A0)
    E0v = S0 @ (np.eye(A0.shape[0]) - P01 @ (I1 - E1v) @ np.linalg.solve(A1, P01.T @ A0)) @ S0
    assert np.abs(E0v - E0).max() > 1e-4


def test_ilut_count_limit_keeps_largest_then_smaller_column():
    """Sec. 4's ILUT, the count limit (reading: keep the ceil(fill * nnz) largest
    |values| of each strictly-lower and strictly-upper row part, exact ties
    going to the smaller column, the diagonal always).  The matrix makes the
    elimination trivial so that the candidates are known by hand: rows 0..7
    hold only their diagonal 1, except row 0 whose upper part is
    (col 3: 2, col 4: -5, col 6: 5, col 7: 2, col 9: -1); row 9 has the lower
    entries (col 1: 3, col 2: -3, col 4: 1, col 5: -4, col 7: 3) and no upper
    part, and every other row only its diagonal.  The pivot rows of row 9
    have no upper entries (and row 0 is not a pivot of row 9), so its
    candidates are its own entries.  With fill = 0.6 the limits are
    ceil(0.6 * 5) = 3 in both row parts."""
    n = 10
    A = np.eye(n) * 4.0
    A[0, [3, 4, 6, 7, 9]] = [2.0, -5.0, 5.0, 2.0, -1.0]
    A[9, [1, 2, 4, 5, 7]] = [3.0, -3.0, 1.0, -4.0, 3.0]
    L, U = pmg.ilut(sp.csr_matrix(A), droptol=0.0, fill=0.6)
    # row 0, upper part: |-5| = |5| (cols 4 and 6), then |2| = |2| tie -> col 3
    u0 = U.getrow(0).toarray().ravel()
    assert sorted(np.nonzero(u0)[0].tolist()) == [0, 3, 4, 6]
    assert u0[4] == -5.0 and u0[6] == 5.0 and u0[3] == 2.0 and u0[0] == 4.0
    # row 9, lower part (pivots are diagonal 4: w_k = a_9k / 4): |-4| (col 5),
    # then the three-way tie |3| = |-3| = |3| at cols 1, 2, 7 -> cols 1 and 2
    l9 = L.getrow(9).toarray().ravel()
    assert sorted(np.nonzero(l9)[0].tolist()) == [1, 2, 5]
    np.testing.assert_array_equal(l9[[1, 2, 5]], [0.75, -0.75, -1.0])
    # the diagonal of row 9 stays: 4, no upper entries
    u9 = U.getrow(9).toarray().ravel()
    assert np.nonzero(u9)[0].tolist() == [9] and u9[9] == 4.0


def test_ilut_on_five_point_laplacian_keeps_the_pattern_of_a():
    """For the 5-point Laplacian every fill-in of the elimination is smaller in
    magnitude than the row's original entries, so with fill = 1 the count
    limit keeps exactly A's pattern in L and U.  (Unlike ILU(0), ILUT uses a
    fill-in pivot before the count limit drops it, so L U does not reproduce
    A on its pattern; the exact-LU and count-limit pins above fix the values.)"""
    A = _grid_laplacian(6).tocsr()
    L, U = pmg.ilut(A, droptol=0.0, fill=1.0)
    low = sp.tril(A, -1).tocsr()
    upp = sp.triu(A, 0).tocsr()
    for M, F in ((low, L), (upp, U)):
        M.sort_indices(); F.sort_indices()
        assert np.array_equal(M.indptr, F.indptr) and np.array_equal(M.indices, F.indices)
    # and dropping did happen: the factors are not the exact LU
    LU = ((sp.identity(A.shape[0]) + L) @ U).toarray()
    assert np.abs(LU - A.toarray()).max() > 1e-3
