"""Pins of the oracle's MGRIT (Sec. 3)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assembly, geometry, mgrit, timestep

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
C = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)


def _problem(p=2, nel=6, geom=None):
    d = assembly.Discretisation(p, nel, geom or geometry.UnitSquare())
    return d, d.project(S), d.load_vector(S)


@pytest.mark.parametrize("Nt,m,ml", [(64, 4, 30), (48, 4, 2), (64, 2, 30), (72, 3, 30)])
def test_fixed_point_is_sequential(Nt, m, ml):
    """The space-time system's unique solution is sequential stepping (its block
    forward solve, Sec. 3)."""
    d, u0, fhat = _problem()
    seq = timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, u0, fhat, C)
    mg = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                     max_levels=ml)
    U, it, hist = mg.run(tol=1e-13, max_iter=60)
    assert hist[-1] <= 1e-13 * hist[0]
    assert np.linalg.norm(U - seq) <= 1e-12 * np.linalg.norm(seq)


def test_single_interval_exact():
    d, u0, fhat = _problem()
    seq = timestep.sequential(d.M, d.K, 1.0, 0.5, 4, u0, fhat, C)
    mg = mgrit.MGRIT(d.M, d.K, 1.0, 0.5, 4, 4, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                     min_coarse=0)
    assert mg.sizes == [4, 1]
    U, it, hist = mg.run(tol=1e-10)
    assert it <= 1
    np.testing.assert_allclose(U, seq, atol=1e-14 * np.abs(seq).max())


@pytest.mark.parametrize("Nt", [60, 62])
@pytest.mark.parametrize("relax,reach", [("F", 1), ("FCF", 2)])
def test_exactness_propagation(relax, reach, Nt):
    """Two-level: after k iterations the first reach*k C-points are exact (also
    with a partial last interval, N_t = 62 = 20 m + 2)."""
    d, u0, fhat = _problem()
    m = 3
    seq = timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, u0, fhat, C)
    for k in (1, 2, 3):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                         max_levels=2, relax=relax)
        U, it, _ = mg.run(tol=0.0, max_iter=k)
        assert it == k
        scale = np.abs(seq).max()
        for j in range(0, reach * k + 1):
            np.testing.assert_allclose(U[j * m], seq[j * m], atol=1e-13 * scale)
        assert np.abs(U[(reach * k + 2) * m] - seq[(reach * k + 2) * m]).max() > 1e-9 * scale


def test_two_level_contraction_bound():
    """Per-iteration contraction of the C-point error (M-norm) against the
    eigenvalue bound of two-level MGRIT theory (Dobrev et al. 2017):
    FCF: |lam|^m |lam^m - lam_c| (1 - |lam_c|^Nc) / (1 - |lam_c|)."""
    d, u0, fhat = _problem(p=2, nel=5)
    kappa, T, Nt, m = 1.0, 2.0, 64, 4
    dt = T / Nt
    mu = sla.eigh(d.K.toarray(), d.M.toarray(), eigvals_only=True)
    lam = 1 / (1 + kappa * dt * mu)
    lamc = 1 / (1 + kappa * m * dt * mu)
    Nc = Nt // m
    bound = np.max(np.abs(lam) ** m * np.abs(lam ** m - lamc) * (1 - np.abs(lamc) ** Nc) / (1 - np.abs(lamc)))
    seq = timestep.sequential(d.M, d.K, kappa, T, Nt, u0, fhat, C)
    Md = d.M.toarray()
    errs = []

    def cb(it, mg):
        e = mg.W[0][::m] - seq[::m]
        errs.append(np.sqrt(sum(v @ Md @ v for v in e)))

    mg = mgrit.MGRIT(d.M, d.K, kappa, T, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                     max_levels=2)
    mg.run(tol=1e-14, max_iter=6, callback=cb)
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    ratios = ratios[np.array(errs[:-1]) > 1e-12 * errs[0]]
    assert len(ratios) >= 2
    assert np.all(ratios <= bound * 1.0001), (ratios, bound)


def test_skip_redundant_F_is_exact_noop():
    d, u0, fhat = _problem()
    a = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, 64, 4, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                    skip_redundant_F=True)
    b = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, 64, 4, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                    skip_redundant_F=False)
    Ua, ia, ha = a.run(tol=0.0, max_iter=3)
    Ub, ib, hb = b.run(tol=0.0, max_iter=3)
    np.testing.assert_allclose(Ua, Ub, rtol=0, atol=1e-15 * np.abs(Ua).max())
    np.testing.assert_allclose(ha, hb, rtol=1e-12)


def test_level_sizes():
    assert mgrit.level_sizes(256, 4) == [256, 64, 16, 4]
    assert mgrit.level_sizes(1024, 8) == [1024, 128, 16, 2]
    assert mgrit.level_sizes(100, 4, max_levels=2) == [100, 25]


def test_level_sizes_ragged():
    """Step counts not divisible by m coarsen to floor(N_l / m) (a partial last
    interval of F-points on the finer level)."""
    assert mgrit.level_sizes(250, 4, min_coarse=2) == [250, 62, 15, 3]
    assert mgrit.level_sizes(7, 4) == [7, 1]
    assert mgrit.level_sizes(3, 4, min_coarse=0) == [3]


@pytest.mark.parametrize("Nt,m,cycle", [(50, 4, "V"), (250, 2, "V"), (61, 3, "F"), (45, 4, "W")])
def test_ragged_fixed_point_is_sequential(Nt, m, cycle):
    """With partial last intervals on several levels the fixed point is still
    sequential stepping, the tail F-points included."""
    d, u0, fhat = _problem()
    seq = timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, u0, fhat, C)
    mg = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                     min_coarse=2, cycle=cycle)
    assert any(s % m for s in mg.sizes[:-1])
    U, it, hist = mg.run(tol=1e-13, max_iter=80)
    assert hist[-1] <= 1e-13 * hist[0]
    assert np.linalg.norm(U - seq) <= 1e-12 * np.linalg.norm(seq)


def test_one_interval_and_tail_exact():
    """N_t = m + 3: one full interval and a tail of three F-points over a
    one-step coarse level; the first correction makes everything exact."""
    d, u0, fhat = _problem()
    seq = timestep.sequential(d.M, d.K, 1.0, 0.5, 7, u0, fhat, C)
    mg = mgrit.MGRIT(d.M, d.K, 1.0, 0.5, 7, 4, mgrit.direct_factory(d.M, d.K), u0, fhat, C)
    assert mg.sizes == [7, 1]
    U, it, hist = mg.run(tol=1e-10)
    assert it <= 1
    np.testing.assert_allclose(U, seq, atol=1e-14 * np.abs(seq).max())


def _paper_iterations():
    """(domain, k, N_t) -> iterations from tests/golden/tables7_8_mgrit_iterations.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tables7_8_mgrit_iterations.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            _, dom, k, nt, it = [f.strip() for f in line.split("|")]
            out[(dom, int(k), int(nt))] = int(it)
    return out


def test_paper_problem_iteration_count_loose():
    """Loose pin on the iteration counts of Tables 7-8 for the paper's problem
    f = 1, u0 = 0, T = 0.1, kappa = 1, tolerance 1e-10, m = 2, min_coarse = 2
    (XBraid's defaults; its other settings are not reproducible here).  The
    paper's counts do not depend on p or h (Table 8), so a coarse mesh (h = 2^-4)
    stands in for h = 2^-6: each count lies within [printed - 2, printed + 1]
    and, like the printed ones, does not decrease as N_t grows."""
    paper = _paper_iterations()
    d = assembly.Discretisation(2, 16, geometry.UnitSquare())
    fhat = d.load_vector(lambda xi, eta, x, y: np.ones_like(x))
    its = []
    for Nt in (100, 250, 500, 1000):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, 0.1, Nt, 2, mgrit.direct_factory(d.M, d.K),
                         np.zeros(d.N), fhat, lambda t: 1.0, min_coarse=2)
        U, it, hist = mg.run(tol=1e-10)
        want = paper[("unit_square", 6, Nt)]
        assert want - 2 <= it <= want + 1, (Nt, it, want)
        its.append(it)
    assert its == sorted(its)


def test_mgrit_with_pmg_solves_matches_sequential():
    hi, lo = assembly.problem(3, 8, geometry.UnitSquare())
    u0 = hi.project(S)
    fhat = hi.load_vector(S)
    seq = timestep.sequential(hi.M, hi.K, 1.0, 1.0, 32, u0, fhat, C)
    mg = mgrit.MGRIT(hi.M, hi.K, 1.0, 1.0, 32, 4, mgrit.pmg_factory(hi, lo, tol=1e-13), u0, fhat, C)
    U, it, hist = mg.run(tol=1e-12)
    assert np.linalg.norm(U - seq) <= 1e-11 * np.linalg.norm(seq)
    assert 0 < np.mean(mg.cycles) < 6


@pytest.mark.parametrize("theta", [0.5, 0.0])
@pytest.mark.parametrize("cycle", ["V", "F", "W"])
def test_theta_and_cycle_fixed_point_is_sequential(theta, cycle):
    """MGRIT's fixed point is sequential theta-stepping for every cycle kind
    (forward Euler on a step small enough to be stable)."""
    d = assembly.Discretisation(2, 4, geometry.UnitSquare())
    u0 = d.project(S)
    fhat = d.load_vector(S)
    c = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)
    T, Nt = (0.5, 64) if theta > 0 else (0.02, 64)
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, u0, fhat, c, theta=theta)
    mg = mgrit.MGRIT(d.M, d.K, 1.0, T, Nt, 4, mgrit.direct_factory(d.M, d.K), u0, fhat, c,
                     theta=theta, cycle=cycle)
    U, it, hist = mg.run(tol=1e-13, max_iter=60)
    assert len(mg.sizes) == 3
    np.testing.assert_allclose(U, seq, rtol=0, atol=1e-11 * np.abs(seq).max())


def test_cycle_kinds_coincide_on_two_levels():
    """With two levels the coarse level is the exact coarsest solve, so V-, F-
    and W-cycles are the same iteration (the repeated visit is skipped)."""
    d = assembly.Discretisation(2, 4, geometry.UnitSquare())
    u0 = d.project(S)
    out = []
    for cycle in ("V", "F", "W"):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, 32, 4, mgrit.direct_factory(d.M, d.K), u0,
                         max_levels=2, cycle=cycle)
        out.append(mg.run(tol=1e-10, max_iter=20))
    for U, it, hist in out[1:]:
        np.testing.assert_array_equal(U, out[0][0])
        assert it == out[0][1] and hist == out[0][2]


def test_f_and_w_cycles_need_no_more_iterations_than_v():
    """More coarse-level work per iteration: on the paper's own problem (f = 1,
    u0 = 0, T = 0.1, Sec. 5) F- and W-cycles converge in at most the
    V-cycle's iterations, and the W-cycle in at most the F-cycle's."""
    d = assembly.Discretisation(2, 8, geometry.UnitSquare())
    fhat = d.load_vector(lambda xi, eta, x, y: np.ones_like(x))
    u0 = np.zeros(d.N)
    its = {}
    for cycle in ("V", "F", "W"):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, 0.1, 256, 2, mgrit.direct_factory(d.M, d.K), u0, fhat,
                         lambda t: 1.0, min_coarse=2, cycle=cycle)
        its[cycle] = mg.run(tol=1e-10, max_iter=50)[1]
    assert its["W"] <= its["F"] <= its["V"], its


def test_inexact_coarse_solves_keep_the_fixed_point():
    """One p-multigrid cycle per coarse-level solve changes the coarse
    propagator only: the converged MGRIT solution is still sequential
    stepping, in the same number of iterations on this problem."""
    from oracle import assembly as asm
    d = asm.Discretisation(2, 8, geometry.UnitSquare())
    lo = asm.Discretisation(1, 8, geometry.UnitSquare())
    u0, fhat = d.project(S), d.load_vector(S)
    c = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)
    seq = timestep.sequential(d.M, d.K, 1.0, 1.0, 64, u0, fhat, c)
    its = []
    for cc in (0, 1):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, 1.0, 64, 4,
                         mgrit.pmg_factory(d, lo, tol=1e-13, coarse_cycles=cc), u0, fhat, c)
        U, it, _ = mg.run(tol=1e-12, max_iter=40)
        np.testing.assert_allclose(U, seq, rtol=0, atol=1e-11 * np.abs(seq).max())
        its.append(it)
    assert its[1] <= its[0] + 1, its
