"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  FP64 form: relative error 1e-10 or better (1e-12 for
single operator products); the mixed form (FP32 smoothing, FP64 refinement)
reaches the same FP64 residual tolerance, so converged solves are held to the
same bound; raw FP32 components to 1e-5."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve, spsolve_triangular

from oracle import assembly, geometry, mgrit, pmg, timestep
from paper_2107_05337_gb300 import inputs

pytestmark = pytest.mark.gpu

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
C = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_05337_gb300 import binding
    binding.lib()
    return binding


def _geom(name):
    return geometry.get(name)


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


CASES = [("unit_square", 2, 8), ("unit_square", 3, 9), ("unit_square", 4, 16),
         ("unit_square", 5, 8), ("quarter_annulus", 2, 8), ("quarter_annulus", 4, 6)]


@pytest.mark.parametrize("geom,p,nel", CASES)
def test_operator_apply_and_vectors(B, geom, p, nel):
    prob = B.Problem(p, nel, geom)
    d = assembly.Discretisation(p, nel, _geom(geom))
    assert prob.N == d.N and prob.n == d.n
    X = inputs.random_block(11, d.N, 5)
    Xd = _cuda(X)
    for which, Mat in (("M", d.M), ("K", d.K)):
        Y = prob.apply(which, Xd).cpu().numpy()
        want = (Mat @ X.T).T
        assert _rel(Y, want) < 1e-13, which
    U0 = lambda xi, eta, x, y: np.sin(np.pi * xi) * np.sin(2 * np.pi * eta) + x * y
    assert _rel(prob.load_vector(U0).cpu().numpy(), d.load_vector(U0)) < 1e-13
    assert _rel(prob.project(U0).cpu().numpy(), d.project(U0)) < 1e-11


def _oracle_pmg(geom, p, nel, c, **kw):
    hi, lo = assembly.problem(p, nel, _geom(geom))
    return hi, pmg.PMG(hi, lo, c, **kw)


@pytest.mark.parametrize("geom,p,nel", [("unit_square", 2, 8), ("unit_square", 3, 9),
                                        ("unit_square", 4, 10), ("quarter_annulus", 3, 8)])
def test_ilut_pattern_bit_exact_and_values(B, geom, p, nel):
    c = 1.0 / 64
    prob = B.Problem(p, nel, geom)
    g = B.PMG(prob, c, precision=0)
    Lg, Ug = g.factors()
    _, P = _oracle_pmg(geom, p, nel, c)
    for G, O in ((Lg, P.L), (Ug, P.U)):
        G.sort_indices(); O.sort_indices()
        assert np.array_equal(G.indptr, O.indptr)
        assert np.array_equal(G.indices, O.indices)
        np.testing.assert_allclose(G.data, O.data, rtol=1e-10, atol=1e-14 * np.abs(O.data).max())
    # level schedule of the pattern (a plain definition) is then identical
    assert np.array_equal(pmg.level_schedule(Lg), pmg.level_schedule(P.L))


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_ilut_block_row_sweeps(B, precision, tol):
    p, nel, c = 4, 12, 1.0 / 128
    prob = B.Problem(p, nel)
    g = B.PMG(prob, c, precision=precision)
    L, U = g.factors()
    R = inputs.random_block(5, prob.N, 7)
    Z = g.ilut_apply(_cuda(R)).cpu().numpy()
    I = sp.identity(prob.N, format="csr")
    for k in range(R.shape[0]):
        y = spsolve_triangular((I + L).tocsr(), R[k], lower=True)
        z = spsolve_triangular(U.tocsr(), y, lower=False)
        assert _rel(Z[k], z) < tol


@pytest.mark.parametrize("geom,p,nel", [("unit_square", 2, 16), ("unit_square", 3, 9),
                                        ("unit_square", 4, 16), ("unit_square", 5, 8),
                                        ("quarter_annulus", 3, 8)])
@pytest.mark.parametrize("ncycles", [1, 2])
def test_pmg_fixed_cycles_fp64(B, geom, p, nel, ncycles):
    """Fixed cycle count: the FP64 GPU cycle equals the oracle's cycle (Sec. 4 steps 1-5)."""
    c = 1.0 / 100
    prob = B.Problem(p, nel, geom)
    g = B.PMG(prob, c, precision=0)
    hi, P = _oracle_pmg(geom, p, nel, c)
    Bm = inputs.random_block(21, prob.N, 4)
    X0 = inputs.random_block(22, prob.N, 4, scale=0.1)
    Xg = _cuda(X0)
    cyc, _ = g.solve(_cuda(Bm), Xg, ncycles=ncycles)
    assert np.all(cyc == ncycles)
    Xg = Xg.cpu().numpy()
    for k in range(Bm.shape[0]):
        x, _ = P.solve(Bm[k], X0[k], ncycles=ncycles)
        assert _rel(Xg[k], x) < 1e-10, k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("geom,p,nel", [("unit_square", 2, 16), ("unit_square", 5, 16),
                                        ("quarter_annulus", 4, 8)])
def test_pmg_converged_vs_direct(B, precision, geom, p, nel):
    c = 1.0 / 64
    prob = B.Problem(p, nel, geom)
    g = B.PMG(prob, c, precision=precision, tol=1e-12)
    d = assembly.Discretisation(p, nel, _geom(geom))
    A = (d.M + c * d.K).tocsc()
    Bm = inputs.random_block(31, prob.N, 6)
    Bm[3] = 0.0                                   # b = 0 gives x = 0 with no cycle
    X = _cuda(np.zeros_like(Bm))
    cyc, _ = g.solve(_cuda(Bm), X)
    X = X.cpu().numpy()
    assert cyc[3] == 0 and np.all(X[3] == 0.0)
    for k in (0, 1, 2, 4, 5):
        x = spsolve(A, Bm[k])
        assert _rel(X[k], x) < 1e-10
        assert np.linalg.norm(Bm[k] - A @ X[k]) <= 1.01e-12 * np.linalg.norm(Bm[k])
        assert 1 <= cyc[k] <= 12


def _oracle_heat(p, nel, T, Nt, geom="unit_square", u0fn=S, source=True):
    d = assembly.Discretisation(p, nel, _geom(geom))
    fhat = d.load_vector(S) if source else None
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(u0fn), fhat, C if source else None)
    return d, seq


def _gpu_heat(B, p, nel, T, Nt, geom="unit_square", u0fn=S, source=True, check=True, **opts):
    prob = B.Problem(p, nel, geom)
    u0 = prob.project(u0fn)
    fhat = prob.load_vector(S) if source else None
    fc = np.array([C(n * T / Nt) for n in range(Nt + 1)]) if source else None
    U, st, status = B.mgrit_solve(prob, u0, fhat, fc, T=T, Nt=Nt, check=check, **opts)
    return U.cpu().numpy(), st


@pytest.mark.parametrize("precision", [0, 1])
def test_mgrit_two_level_c1_shape(B, precision):
    """Config shape c1 (p=2, 16 elements, N_t=100, two-level, m=4, FCF): the
    converged GPU MGRIT equals sequential backward Euler (Sec. 3)."""
    d, seq = _oracle_heat(2, 16, 1.0, 100)
    U, st = _gpu_heat(B, 2, 16, 1.0, 100, m=4, max_levels=2, tol=1e-12,
                      pmg=dict(tol=1e-13, precision=precision))
    assert st["levels"] == 2
    assert _rel(U, seq) < 1e-10, st
    assert 5 <= st["iters"] <= 15


def test_mgrit_fixed_iterations_match_oracle(B):
    """Fixed MGRIT iteration count (2 and 3), FP64, tight spatial tolerance:
    the GPU iterate equals the oracle MGRIT iterate of the same schedule."""
    p, nel, T, Nt, m = 3, 8, 1.0, 48, 4
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    u0, fhat = d.project(S), d.load_vector(S)
    for k in (1, 2, 3):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, T, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C)
        Uo, it, hist = mg.run(tol=0.0, max_iter=k)
        # tol = 0 forces exactly k iterations; the call then reports NOT_CONVERGED
        U, st = _gpu_heat(B, p, nel, T, Nt, check=False, m=m, tol=0.0, max_iter=k,
                          pmg=dict(tol=1e-14, precision=0, max_cycles=60))
        assert st["iters"] == k
        assert _rel(U, Uo) < 1e-10, k
        np.testing.assert_allclose(st["res_hist"], hist, rtol=1e-8)


@pytest.mark.parametrize("relax", [0, 1])
def test_mgrit_multilevel_and_relaxation(B, relax):
    d, seq = _oracle_heat(3, 16, 1.0, 64)
    U, st = _gpu_heat(B, 3, 16, 1.0, 64, m=4, relax=relax, tol=1e-12, max_iter=60,
                      pmg=dict(tol=1e-13, precision=1))
    assert st["levels"] == 3
    assert _rel(U, seq) < 1e-10, st


def test_mgrit_curved_annulus(B):
    k, l, a = inputs.fourier_modes()
    u0fn = lambda xi, eta, x, y: sum(a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta)
                                     for s in range(len(a)))
    d, seq = _oracle_heat(3, 8, 1.0, 64, "quarter_annulus", u0fn, source=False)
    U, st = _gpu_heat(B, 3, 8, 1.0, 64, "quarter_annulus", u0fn, source=False, m=8, tol=1e-12,
                      pmg=dict(tol=1e-13, precision=1))
    assert st["levels"] == 3
    assert _rel(U, seq) < 1e-10, st


def test_mgrit_nt_equals_m_and_sequential_fallback(B):
    d, seq = _oracle_heat(2, 8, 0.5, 4)
    U, st = _gpu_heat(B, 2, 8, 0.5, 4, m=4, min_coarse=0, tol=1e-12, pmg=dict(tol=1e-13))
    assert st["iters"] <= 1 and _rel(U, seq) < 1e-10
    # N_t = m + 3: one interval and a partial last interval of three F-points
    # over a one-step coarse level: exact after the first correction
    d, seq = _oracle_heat(2, 8, 0.5, 7)
    U, st = _gpu_heat(B, 2, 8, 0.5, 7, m=4, tol=1e-12, pmg=dict(tol=1e-13))
    assert st["levels"] == 2 and st["iters"] <= 1 and _rel(U, seq) < 1e-10
    # fewer steps than m: no coarse level, plain sequential stepping
    d, seq = _oracle_heat(2, 8, 0.5, 3)
    U, st = _gpu_heat(B, 2, 8, 0.5, 3, m=4, min_coarse=0, tol=1e-12, pmg=dict(tol=1e-13))
    assert st["levels"] == 1 and _rel(U, seq) < 1e-10


def test_mgrit_ragged_fixed_iterations_match_oracle(B):
    """Step counts that m does not divide (N_t = 50, m = 4: levels 50, 12, 3,
    a partial last interval on the fine level): fixed iterations, FP64, tight
    spatial tolerance, against the oracle iterate and residual history."""
    p, nel, T, Nt, m = 2, 8, 1.0, 50, 4
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    u0, fhat = d.project(S), d.load_vector(S)
    for k in (1, 2):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, T, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                         min_coarse=2)
        assert mg.sizes == [50, 12, 3]
        Uo, it, hist = mg.run(tol=0.0, max_iter=k)
        U, st = _gpu_heat(B, p, nel, T, Nt, check=False, m=m, min_coarse=2, tol=0.0, max_iter=k,
                          pmg=dict(tol=1e-14, precision=0, max_cycles=60))
        assert st["levels"] == 3 and st["iters"] == k
        assert _rel(U, Uo) < 1e-10, k
        np.testing.assert_allclose(st["res_hist"], hist, rtol=1e-8)


@pytest.mark.parametrize("Nt,m,cycle", [(250, 2, 0), (99, 4, 2)])
def test_mgrit_ragged_converged(B, Nt, m, cycle):
    """Partial last intervals on several levels (N_t = 250, m = 2: seven
    levels; N_t = 99, m = 4 with W-cycles), mixed form, against sequential
    stepping."""
    d, seq = _oracle_heat(2, 8, 1.0, Nt)
    U, st = _gpu_heat(B, 2, 8, 1.0, Nt, m=m, min_coarse=2, cycle=cycle, tol=1e-12, max_iter=60,
                      pmg=dict(tol=1e-13, precision=1))
    assert st["levels"] == len(mgrit.level_sizes(Nt, m, min_coarse=2))
    assert _rel(U, seq) < 1e-10, st


def test_invalid_arguments_raise(B):
    with pytest.raises(B.IgmError):
        B.Problem(1, 8)
    prob = B.Problem(2, 8)
    with pytest.raises(B.IgmError):
        B.PMG(prob, 0.01, nu1=0, nu2=0)
    with pytest.raises(B.IgmError):
        B.PMG(prob, 0.01, precision=3)
