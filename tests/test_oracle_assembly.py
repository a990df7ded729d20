"""Pins of the oracle's assembly (Sec. 2 matrices, Sec. 4 transfer and lumping)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import assembly, bspline, geometry
from stencil_rows import unit_square_row


def test_q1_textbook_stencils():
    """p = 1 is the low-order Lagrange (Q1) discretisation (Sec. 4)."""
    nel = 6
    h = 1.0 / nel
    d = assembly.Discretisation(1, nel, geometry.UnitSquare())
    nb = d.nb
    i = 3 + nb * 3                                    # an interior node
    M = d.M_full.toarray()[i].reshape(nb, nb)[2:5, 2:5]
    K = d.K_full.toarray()[i].reshape(nb, nb)[2:5, 2:5]
    np.testing.assert_allclose(M, h * h / 36 * np.array([[1, 4, 1], [4, 16, 4], [1, 4, 1]]), atol=1e-16)
    np.testing.assert_allclose(K, 1 / 3 * np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]), atol=1e-14)


@pytest.mark.parametrize("p,nel", [(1, 4), (2, 5), (3, 4), (4, 3), (5, 2)])
def test_unit_square_mass_sum_stiffness_rowsum_lumping(p, nel):
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    assert abs(d.M_full.sum() - 1.0) < 1e-13
    assert np.abs(np.asarray(d.K_full.sum(axis=1))).max() < 1e-12
    # closed-form lumped mass on the unit square: prod_d (xi_{i+p+1}-xi_i)/(p+1)
    t = d.knots
    one_d = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(d.nb)])
    np.testing.assert_allclose(d.lumped_full, np.kron(one_d, one_d), rtol=1e-13)


@pytest.mark.parametrize("p", [2, 4])
def test_annulus_area_symmetry_definiteness(p):
    g = geometry.QuarterAnnulus()
    d = assembly.Discretisation(p, 4, g)
    assert abs(d.M_full.sum() - g.area_by_green()) < 1e-12
    # exact circle would give 3 pi / 4; the cubic arc is within 3e-4 of it
    assert abs(g.area_by_green() - 0.75 * np.pi) < 3e-3
    assert np.abs(np.asarray(d.K_full.sum(axis=1))).max() < 1e-11
    for A in (d.M, d.K):
        Ad = A.toarray()
        np.testing.assert_allclose(Ad, Ad.T, atol=1e-14 * np.abs(Ad).max())
        assert np.linalg.eigvalsh(Ad).min() > 0


def test_transfer_reproduces_constants():
    """Partition of unity + row-sum lumping: (M_p^L)^{-1} P 1 = 1 and
    (M_1^L)^{-1} P^T 1 = 1 on the full bases (Sec. 4)."""
    for geom in (geometry.UnitSquare(), geometry.QuarterAnnulus()):
        hi, lo = assembly.problem(3, 5, geom)
        P = hi.transfer_to(lo, full=True)
        np.testing.assert_allclose(P @ np.ones(P.shape[1]) / hi.lumped_full, 1.0, rtol=1e-12)
        np.testing.assert_allclose(P.T @ np.ones(P.shape[0]) / lo.lumped_full, 1.0, rtol=1e-12)


def test_dirichlet_sizes():
    for p, nel, N in [(2, 16, 256), (4, 128, 16900), (3, 64, 4225)]:
        knots = bspline.open_uniform_knots(p, nel)
        n = bspline.num_basis(knots, p) - 2
        assert n * n == N


@pytest.mark.parametrize("p,nel", [(2, 23), (3, 19), (5, 25)])
def test_unit_square_rows_translate_and_scale(p, nel):
    """On the unit square with open uniform knots (Sec. 2) every row of M and K
    whose coupled basis functions have uniform knot spans is one translated
    stencil; M scales with h^2 and K not at all; rows near an edge repeat those
    of a small problem at the same distance from the edge.  Every row of the
    oracle's nel x nel matrices against the rows mapped from a (4p + 2)^2
    problem: a wrong quadrature weight, basis index or Jacobian factor in the
    assembly breaks the relation."""
    nel_s = 4 * p + 2
    ds = assembly.Discretisation(p, nel_s, geometry.UnitSquare())
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    n = d.n
    for iy in range(n):
        for ix in range(n):
            st = unit_square_row(ds, nel_s, nel, p, n, iy, ix)
            r = iy * n + ix
            for k, mat in enumerate((d.M, d.K)):
                row = mat.getrow(r)
                got = {(j // n - iy, j % n - ix): v for j, v in zip(row.indices, row.data)}
                scale = np.abs(row.data).max()
                for key in set(got) | set(st):
                    assert abs(got.get(key, 0.0) - st.get(key, (0.0, 0.0))[k]) <= 1e-12 * scale
