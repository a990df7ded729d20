"""Pins of the oracle's Jacobi-preconditioned CG (the paper's comparison solver, Sec. 5)."""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from oracle import assembly, cg, geometry


def _krylov_minimiser(A, b, x0, k):
    """argmin over x0 + K_k(D^-1 A, D^-1 r0) of the A-norm error, by projection."""
    A = A.toarray()
    dinv = 1.0 / np.diag(A)
    r0 = b - A @ x0
    V = [dinv * r0]
    for _ in range(k - 1):
        V.append(dinv * (A @ V[-1]))
    V = np.array(V).T
    Q, _ = np.linalg.qr(V)
    y = np.linalg.solve(Q.T @ A @ Q, Q.T @ r0)
    return x0 + Q @ y


def test_iterates_minimise_energy_error_over_krylov_space():
    d = assembly.Discretisation(3, 3, geometry.QuarterAnnulus())
    A = (d.M + 0.02 * d.K).tocsr()
    rng = np.random.default_rng(5)
    b = rng.standard_normal(d.N)
    x0 = rng.standard_normal(d.N)
    for k in (1, 2, 4, 7):
        x, it = cg.pcg_jacobi(A, b, x0, niter=k)
        assert it == k
        want = _krylov_minimiser(A, b, x0, k)
        np.testing.assert_allclose(x, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_diagonal_matrix_one_iteration():
    a = np.array([1.0, 3.0, 0.5, 7.0])
    b = np.array([2.0, -1.0, 4.0, 0.25])
    x, it = cg.pcg_jacobi(sp.diags(a), b, tol=1e-14)
    assert it == 1
    np.testing.assert_allclose(x, b / a, rtol=1e-15)


def test_converges_to_direct_solve():
    d = assembly.Discretisation(4, 8, geometry.UnitSquare())
    A = (d.M + 0.01 * d.K).tocsr()
    b = np.random.default_rng(2).standard_normal(d.N)
    x, it = cg.pcg_jacobi(A, b, tol=1e-12)
    np.testing.assert_allclose(x, spsolve(A.tocsc(), b), rtol=1e-9, atol=1e-11)


def test_iterations_grow_with_p():
    """Fixed h = 1/16, A = M + 1/256 K: CG needs more iterations at higher p
    (the p-dependence that motivates p-multigrid, Sec. 4-5)."""
    its = []
    for p in (2, 3, 4, 5):
        d = assembly.Discretisation(p, 16, geometry.UnitSquare())
        A = (d.M + d.K / 256.0).tocsr()
        b = d.load_vector(lambda xi, eta, x, y: np.ones_like(x))
        its.append(cg.pcg_jacobi(A, b, tol=1e-10)[1])
    assert all(b > a for a, b in zip(its, its[1:])), its
