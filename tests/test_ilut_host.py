"""The library's host ILUT (pmg_ilut_host: the factorisation pmg_setup runs,
Sec. 4's smoother) against the oracle's ILUT on the same matrices: patterns
and values bit-exact (both eliminate in the same order with one rounding per
operation).  Runs on the CPU: the call needs no device."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly, geometry, pmg


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding, build
    build.build()
    return binding


def _same(G, O):
    G, O = G.tocsr(), O.tocsr()
    G.sort_indices()
    O.sort_indices()
    return (np.array_equal(G.indptr, O.indptr) and np.array_equal(G.indices, O.indices)
            and np.array_equal(G.data, O.data))


@pytest.mark.parametrize("geom,p,nel", [(geometry.UnitSquare, 2, 8), (geometry.UnitSquare, 3, 9),
                                        (geometry.UnitSquare, 4, 10), (geometry.UnitSquare, 5, 8),
                                        (geometry.QuarterAnnulus, 3, 8)])
def test_iga_matrices_bit_exact(B, geom, p, nel):
    hi, lo = assembly.problem(p, nel, geom())
    for c in (1.0 / 64, 1.0):
        P = pmg.PMG(hi, lo, c)
        L, U = B.ilut_host(P.A)
        assert _same(L, P.L) and _same(U, P.U)


@pytest.mark.parametrize("droptol,fill", [(1e-12, 1.0), (1e-2, 1.0), (1e-3, 0.5), (0.0, 3.0)])
def test_random_pattern_bit_exact(B, droptol, fill):
    """A diagonally dominant random sparse matrix (no tensor-product
    structure), with dropping and the entry limits both active."""
    rng = np.random.default_rng(5)
    n = 60
    R = sp.random(n, n, density=0.08, random_state=rng, format="csr")
    A = (R + R.T + sp.diags(np.abs(R).sum(axis=1).A1 + np.abs(R).sum(axis=0).A1 + 1.0)).tocsr()
    A.sort_indices()
    Lo, Uo = pmg.ilut(A, droptol, fill)
    L, U = B.ilut_host(A, droptol, fill)
    assert _same(L, Lo) and _same(U, Uo)


def test_no_dropping_is_exact_lu(B):
    hi, lo = assembly.problem(2, 6, geometry.UnitSquare())
    A = (hi.M + 0.1 * hi.K).tocsr()
    L, U = B.ilut_host(A, 0.0, 1e6)
    Lu = (sp.identity(A.shape[0]) + L) @ U
    assert abs(Lu - A).max() <= 1e-13 * abs(A).max()


def test_errors(B):
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))
    with pytest.raises(B.IgmError):        # zero pivot in row 0
        B.ilut_host(A)
    with pytest.raises(B.IgmError):        # negative drop tolerance
        B.ilut_host(sp.identity(3, format="csr"), droptol=-1.0)


@pytest.mark.parametrize("geom,p,nel", [(geometry.UnitSquare, 3, 8), (geometry.QuarterAnnulus, 4, 6)])
def test_block_row_form_of_the_factors(B, geom, p, nel):
    """pmg_block_tri_host (the data the ILUT sweeps stream): the couplings to
    other grid rows plus the diagonal blocks give back the factor exactly, and
    each packed inverse is the inverse of its (unit-)triangular diagonal block."""
    hi, lo = assembly.problem(p, nel, geom())
    P = pmg.PMG(hi, lo, 1.0 / 64)
    L, U = B.ilut_host(P.A)
    n = hi.n
    N = n * n
    for F, upper in ((L, False), (U, True)):
        off, inv = B.block_tri_host(F, n, upper)
        D = sp.lil_matrix((N, N))
        dense = F.toarray()
        for b in range(n):
            s = slice(b * n, (b + 1) * n)
            blk = dense[s, s] + (0.0 if upper else np.eye(n))
            I = inv[b] @ blk
            assert np.abs(I - np.eye(n)).max() <= 1e-10, (upper, b)
            D[s, s] = dense[s, s]
        assert abs(off + D.tocsr() - F).max() == 0.0
        assert all(c // n != r // n for r in range(N) for c in off.indices[off.indptr[r]:off.indptr[r + 1]])


def test_block_row_form_rejects_entries_outside_the_triangle(B):
    F = sp.csr_matrix(np.triu(np.ones((4, 4))))      # n = 2: an upper factor passed as lower
    with pytest.raises(B.IgmError):
        B.block_tri_host(F, 2, upper=False)
