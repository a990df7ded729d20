"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (one MGRIT handle per problem, concurrent-safe streams), against
the oracle's sequential backward Euler with direct solves; plus the failure
detection self-test.  These are the slow GPU tests (about a minute)."""
import numpy as np
import pytest

from oracle import assembly, geometry, timestep
from paper_2107_05337_gb300 import inputs

pytestmark = pytest.mark.gpu

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
C = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding
    binding.lib()
    return binding


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_wait_selftest_times_out_and_device_stays_usable(B):
    """A bounded mbarrier wait on a barrier nothing completes returns
    IGM_ERR_TIMEOUT; the context then still runs a solve."""
    assert B.wait_selftest(1 << 12) == -5
    assert "gave up" in B.lib().igm_last_error().decode()
    prob = B.Problem(2, 8)
    u0 = prob.project(S)
    U, st, status = B.mgrit_solve(prob, u0, T=0.25, Nt=8, m=4, tol=1e-10)
    assert status == 0 and st["iters"] >= 1


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_heat_c2_full_size(B, p):
    """Unit square, 64 x 64 elements, N_t = 256, m = 4, 256 -> 64 -> 16 -> 4.
    Bench tolerances (1e-10; the mixed and FP64 forms, and the benchmarked form
    with one cycle per coarse-level solve and autotuned sweep layouts): error
    vs sequential BE within the tolerance-stacking bound 5e-10 (a solution
    converged to a 1e-10 residual is that close, not closer); tight
    tolerances (MGRIT 1e-12, spatial 1e-13), both forms: within 1e-10."""
    nel, T, Nt = 64, 1.0, 256
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C)
    prob = B.Problem(p, nel)
    u0, fhat = prob.project(S), prob.load_vector(S)
    fc = np.array([C(n * T / Nt) for n in range(Nt + 1)])
    forms = ((dict(precision=1, tol=1e-10), {}), (dict(precision=0, tol=1e-10), {}),
             (dict(precision=1, tol=1e-10, autotune=1), dict(coarse_cycles=1)))
    for pmg_opts, extra in forms:
        mg = B.MGRIT(prob, T=T, Nt=Nt, m=4, tol=1e-10, pmg=pmg_opts, **extra)
        U, st, _ = mg.run(u0, fhat, fc)
        assert st["levels"] == 4 and 7 <= st["iters"] <= 12
        assert _rel(U.cpu().numpy(), seq) < 5e-10, (pmg_opts, extra, st)
    for precision in (1, 0):      # tight tolerances: both forms within 1e-10
        mg = B.MGRIT(prob, T=T, Nt=Nt, m=4, tol=1e-12, pmg=dict(precision=precision, tol=1e-13))
        U, st, _ = mg.run(u0, fhat, fc)
        assert _rel(U.cpu().numpy(), seq) < 1e-10, (precision, st)


def test_annulus_c3_full_size(B):
    """Quarter annulus, p = 4, 128 x 128 elements (N = 16900), N_t = 1024,
    m = 8 (1024 -> 128 -> 16 -> 2), f = 0, 8-mode Fourier initial condition."""
    p, nel, T, Nt = 4, 128, 1.0, 1024
    k, l, a = inputs.fourier_modes()
    u0fn = lambda xi, eta, x, y: sum(a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta)
                                     for s in range(len(a)))
    d = assembly.Discretisation(p, nel, geometry.QuarterAnnulus())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(u0fn))
    prob = B.Problem(p, nel, "quarter_annulus")
    assert prob.N == 16900
    u0 = prob.project(u0fn)
    # the mixed form, and the benchmarked form (one cycle per coarse-level
    # solve, autotuned sweep layouts), at bench tolerances
    forms = ((dict(precision=1, tol=1e-10), {}),
             (dict(precision=1, tol=1e-10, autotune=1), dict(coarse_cycles=1)))
    for pmg_opts, extra in forms:
        mg = B.MGRIT(prob, T=T, Nt=Nt, m=8, tol=1e-10, pmg=pmg_opts, **extra)
        U, st, _ = mg.run(u0)
        assert st["levels"] == 4
        assert _rel(U.cpu().numpy(), seq) < 5e-10, (pmg_opts, extra, st)
    # the FP64 form at tight tolerances: within 1e-10
    mg = B.MGRIT(prob, T=T, Nt=Nt, m=8, tol=1e-12, pmg=dict(precision=0, tol=1e-13))
    U, st, _ = mg.run(u0)
    assert _rel(U.cpu().numpy(), seq) < 1e-10, st


def test_grid_barrier_selftest_times_out_and_device_stays_usable(B):
    """The grid-wide barrier of a fused level visit (one cooperative launch for
    the F, C and F + residual phases): all CTAs pass it; when one CTA holds
    back (a host-set flag), every wait gives up after its bound, the call
    returns IGM_ERR_TIMEOUT, and the context still runs a fused solve."""
    assert B.grid_barrier_selftest(nctas=16, hold=0) == 0
    assert B.grid_barrier_selftest(nctas=16, wait_cycles=1 << 22, hold=1) == -5
    assert "gave up" in B.lib().igm_last_error().decode()
    prob = B.Problem(2, 8)
    u0 = prob.project(S)
    U, st, status = B.mgrit_solve(prob, u0, T=0.25, Nt=16, m=4, tol=1e-10, fused=1)
    assert status == 0 and st["iters"] >= 1


@pytest.mark.parametrize("p,precision", [(3, 0), (4, 1)])
def test_fused_level_visits_equal_separate_launches(B, p, precision):
    """Fused level visits (one cooperative launch per visit, grid barriers
    between the phases) give bit-identical iterates, iteration counts and
    residual histories to one launch per phase (Sec. 3's FCF relaxation),
    on a level count with a partial interval, with and without graphs; and
    fewer kernel launches."""
    nel, T, Nt = 16, 1.0, 100
    prob = B.Problem(p, nel)
    u0, fhat = prob.project(S), prob.load_vector(S)
    fc = np.array([C(n * T / Nt) for n in range(Nt + 1)])
    out = {}
    for fused in (0, 1):
        for graphs in (0, 1):
            mg = B.MGRIT(prob, T=T, Nt=Nt, m=4, tol=1e-10, fused=fused, graphs=graphs,
                         pmg=dict(precision=precision, tol=1e-10))
            U, st, _ = mg.run(u0, fhat, fc)
            out[(fused, graphs)] = (U.cpu().numpy(), st)
    ref_U, ref_st = out[(0, 0)]
    for key, (U, st) in out.items():
        assert np.array_equal(U, ref_U), key
        assert st["iters"] == ref_st["iters"], key
        assert np.array_equal(np.asarray(st["res_hist"]), np.asarray(ref_st["res_hist"])), key
    assert out[(1, 1)][1]["launches"] < out[(0, 1)][1]["launches"]
