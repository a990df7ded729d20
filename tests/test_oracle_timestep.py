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
