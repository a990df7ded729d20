"""Pins of the oracle's sequential backward Euler (Sec. 2 Eq. (los), theta=1)."""
import numpy as np
import scipy.linalg as sla

from oracle import assembly, geometry, timestep

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)


def test_generalised_eigenvector_decay_exact():
    d = assembly.Discretisation(2, 5, geometry.UnitSquare())
    mu, V = sla.eigh(d.K.toarray(), d.M.toarray())
    kappa, T, Nt = 1.7, 0.3, 12
    dt = T / Nt
    for k in (0, 7, len(mu) - 1):
        U = timestep.sequential(d.M, d.K, kappa, T, Nt, V[:, k])
        for n in range(Nt + 1):
            np.testing.assert_allclose(U[n], (1 + kappa * dt * mu[k]) ** (-n) * V[:, k],
                                       rtol=1e-10, atol=1e-12 * np.abs(V[:, k]).max())


def test_step_matches_dense_solve():
    d = assembly.Discretisation(3, 3, geometry.QuarterAnnulus())
    rng = np.random.default_rng(1)
    u = rng.standard_normal(d.N)
    f = rng.standard_normal(d.N)
    be = timestep.BackwardEuler(d.M, d.K, 0.5, 0.01)
    A = d.M.toarray() + 0.5 * 0.01 * d.K.toarray()
    want = np.linalg.solve(A, d.M.toarray() @ u + 0.01 * f)
    np.testing.assert_allclose(be.step(u, f), want, rtol=1e-12, atol=1e-13)


def test_manufactured_first_order_in_time():
    """u = sin(pi x) sin(pi y) cos t, f = (2 pi^2 cos t - sin t) sin(pi x) sin(pi y):
    with the spatial error negligible, the error at T halves with dt."""
    d = assembly.Discretisation(4, 8, geometry.UnitSquare())
    u0 = d.project(S)
    fhat = d.load_vector(S)
    c = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)
    exact = lambda xi, eta, x, y: S(xi, eta, x, y) * np.cos(1.0)
    errs = [d.l2_error(timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, u0, fhat, c)[-1], exact)
            for Nt in (20, 40, 80)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 1.0) < 0.1), rates


def test_theta_eigenvector_decay_exact():
    """Eq. (los) on K v = mu M v: u_n = ((1-(1-theta) k dt mu)/(1+theta k dt mu))^n v."""
    d = assembly.Discretisation(2, 5, geometry.UnitSquare())
    mu, V = sla.eigh(d.K.toarray(), d.M.toarray())
    kappa, T, Nt = 0.7, 0.05, 10
    dt = T / Nt
    for theta in (0.5, 0.0, 0.3):
        for k in (0, 5, len(mu) - 1):
            U = timestep.sequential(d.M, d.K, kappa, T, Nt, V[:, k], theta=theta)
            g = (1 - (1 - theta) * kappa * dt * mu[k]) / (1 + theta * kappa * dt * mu[k])
            for n in range(Nt + 1):
                np.testing.assert_allclose(U[n], g ** n * V[:, k], rtol=1e-9,
                                           atol=1e-11 * max(1.0, abs(g) ** n) * np.abs(V[:, k]).max())


def _semidiscrete_exact(d, kappa, T, u0, fhat, c):
    """Exact solution at T of M u' + kappa K u = c(t) fhat, u(0) = u0, by the
    generalised eigen-decomposition (V^T M V = I) and composite Gauss-Legendre
    quadrature of the source integral."""
    mu, V = sla.eigh(d.K.toarray(), d.M.toarray())
    a0 = V.T @ (d.M @ u0)
    b = V.T @ fhat
    x, w = np.polynomial.legendre.leggauss(20)
    integ = np.zeros_like(mu)
    edges = np.linspace(0.0, T, 201)
    for lo, hi in zip(edges[:-1], edges[1:]):
        s = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        for si, wi in zip(s, w):
            integ += 0.5 * (hi - lo) * wi * np.exp(-kappa * mu * (T - si)) * c(si)
    return V @ (np.exp(-kappa * mu * T) * a0 + integ * b)


def test_theta_scheme_order_against_semidiscrete_solution():
    """Backward Euler is first and Crank-Nicolson second order in dt against
    the exact solution of the semi-discrete system (no spatial error)."""
    d = assembly.Discretisation(2, 3, geometry.UnitSquare())
    u0 = d.project(S)
    fhat = d.load_vector(S)
    c = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)
    ref = _semidiscrete_exact(d, 1.0, 1.0, u0, fhat, c)
    for theta, order in ((1.0, 1.0), (0.5, 2.0)):
        errs = [np.linalg.norm(timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, u0, fhat, c,
                                                   theta=theta)[-1] - ref)
                for Nt in (40, 80, 160)]
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all(np.abs(rates - order) < 0.1), (theta, rates)
