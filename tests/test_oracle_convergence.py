"""Discretisation accuracy pins: O(h^{p+1}) L2 convergence (IgA with B-splines
of order p on a uniform mesh, Sec. 2)."""
import numpy as np
import pytest
from scipy.sparse.linalg import spsolve

from oracle import assembly, geometry

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_l2_projection_rate(p):
    errs = []
    for nel in (8, 16, 32):
        d = assembly.Discretisation(p, nel, geometry.UnitSquare())
        errs.append(d.l2_error(d.project(S), S))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - (p + 1)) < 0.15, rates


@pytest.mark.parametrize("p", [2, 3])
def test_poisson_rate(p):
    """-Delta u = 2 pi^2 sin(pi x) sin(pi y), u = sin(pi x) sin(pi y): K u = b."""
    errs = []
    for nel in (8, 16, 32):
        d = assembly.Discretisation(p, nel, geometry.UnitSquare())
        b = d.load_vector(lambda xi, eta, x, y: 2 * np.pi ** 2 * S(xi, eta, x, y))
        u = spsolve(d.K.tocsc(), b)
        errs.append(d.l2_error(u, S))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - (p + 1)) < 0.15, rates


def test_poisson_rate_annulus():
    """Manufactured solution on the curved map: u = sin(pi xi) sin(pi eta) pulled
    back; check convergence of the projection at rate p+1 (p=2)."""
    g = geometry.QuarterAnnulus()
    U = lambda xi, eta, x, y: np.sin(np.pi * xi) * np.sin(np.pi * eta)
    errs = []
    for nel in (8, 16, 32):
        d = assembly.Discretisation(2, nel, g)
        errs.append(d.l2_error(d.project(U), U))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - 3) < 0.15, rates
