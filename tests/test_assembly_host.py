"""The library's host assembly (iga_assemble_host: the matrices iga_assemble
uploads; Sec. 2) against the oracle's independent assembly: M, K and the
lumped masses on the unit square and on the curved quarter annulus, to FP64
rounding (the two sum the quadrature in different orders).  Runs on the CPU:
the call needs no device."""
import numpy as np
import pytest

from oracle import assembly, geometry, pmg


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("geom,G", [("unit_square", geometry.UnitSquare),
                                    ("quarter_annulus", geometry.QuarterAnnulus)])
@pytest.mark.parametrize("p,nel", [(1, 5), (2, 4), (3, 7), (4, 6), (5, 5)])
def test_host_assembly_matches_oracle(B, geom, G, p, nel):
    d = assembly.Discretisation(p, nel, G())
    for which, A in (("M", d.M), ("K", d.K)):
        H = B.assemble_host(p, nel, geom, which)
        assert H.shape == A.shape
        assert abs(H - A).max() <= 1e-13 * abs(A).max(), which
        # same sparsity: every stencil coupling inside the grid is structurally nonzero
        assert (abs(H) > 0).nnz == (abs(A) > 0).nnz
    lum = B.assemble_host(p, nel, geom, "lumped")
    assert np.abs(lum - d.lumped).max() <= 1e-13 * np.abs(d.lumped).max()


def test_invalid_arguments(B):
    with pytest.raises(B.IgmError):
        B.assemble_host(0, 4)
    with pytest.raises(ValueError):
        B.assemble_host(2, 4, "disk")


@pytest.mark.parametrize("geom,G", [("unit_square", geometry.UnitSquare),
                                    ("quarter_annulus", geometry.QuarterAnnulus)])
@pytest.mark.parametrize("p,nel", [(2, 4), (3, 7), (5, 6)])
def test_host_transfer_matches_oracle(B, geom, G, p, nel):
    """The order-p x order-1 transfer matrix P of Eq. (PM), interior x interior."""
    hi, lo = assembly.problem(p, nel, G())
    O = hi.transfer_to(lo)
    H = B.transfer_host(p, nel, geom)
    assert H.shape == O.shape
    assert (abs(H) > 0).nnz == (abs(O) > 0).nnz
    assert abs(H - O).max() <= 1e-13 * abs(O).max()


@pytest.mark.parametrize("geom,G", [("unit_square", geometry.UnitSquare),
                                    ("quarter_annulus", geometry.QuarterAnnulus)])
@pytest.mark.parametrize("p,nel,coarsest", [(2, 32, 8), (4, 16, 8), (3, 24, 4), (2, 12, 8)])
def test_host_h_hierarchy_matches_oracle(B, geom, G, p, nel, coarsest):
    """The order-1 operator and its Galerkin h-levels (Sec. 4, Fig. 5): the same
    number of levels (coarsening while the element count is even and above the
    coarsest) and the same operators as the oracle's P^T A P."""
    hi, lo = assembly.problem(p, nel, G())
    c = 1.0 / 64
    O = pmg.HMG((lo.M + c * lo.K).tocsr(), nel, coarsest).A
    H = B.hmg_host(p, nel, c, geom, coarsest)
    assert len(H) == len(O)
    for h, o in zip(H, O):
        assert h.shape == o.shape
        assert abs(h - o).max() <= 1e-13 * abs(o).max()
