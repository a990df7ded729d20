"""GPU parity of the method variants: the theta-scheme of Sec. 2 Eq. (los)
(Crank-Nicolson, forward Euler beside backward Euler) and the MGRIT F- and
W-cycles named in Sec. 5, against the CPU oracle on the same inputs."""
import numpy as np
import pytest

from oracle import assembly, geometry, mgrit, timestep
from stencil_rows import unit_square_row

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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _gpu(B, p, nel, T, Nt, check=True, geom="unit_square", **opts):
    prob = B.Problem(p, nel, geom)
    u0, fhat = prob.project(S), prob.load_vector(S)
    fc = np.array([C(n * T / Nt) for n in range(Nt + 1)])
    U, st, status = B.mgrit_solve(prob, u0, fhat, fc, T=T, Nt=Nt, check=check, **opts)
    return U.cpu().numpy(), st


@pytest.mark.parametrize("cycle", ["V", "F", "W"])
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_fixed_iterations_match_oracle(B, theta, cycle):
    """k MGRIT iterations (FP64 form, tight spatial tolerance) with four time
    levels: the GPU iterate and residual history equal the oracle's."""
    p, nel, T, Nt, m = 2, 8, 1.0, 128, 4
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    u0, fhat = d.project(S), d.load_vector(S)
    for k in (1, 2):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, T, Nt, m, mgrit.direct_factory(d.M, d.K), u0, fhat, C,
                         theta=theta, cycle=cycle)
        Uo, it, hist = mg.run(tol=0.0, max_iter=k)
        assert len(mg.sizes) == 4
        U, st = _gpu(B, p, nel, T, Nt, check=False, m=m, tol=0.0, max_iter=k, theta=theta,
                     cycle=cycle, pmg=dict(tol=1e-14, precision=0, max_cycles=60))
        assert st["iters"] == k and st["levels"] == 4
        assert _rel(U, Uo) < 1e-10, (theta, cycle, k)
        np.testing.assert_allclose(st["res_hist"], hist, rtol=1e-8)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("cycle", ["V", "F"])
def test_crank_nicolson_converges_to_sequential(B, precision, cycle):
    """Converged MGRIT with Crank-Nicolson steps equals sequential CN stepping."""
    p, nel, T, Nt = 3, 16, 1.0, 64
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C, theta=0.5)
    U, st = _gpu(B, p, nel, T, Nt, m=4, tol=1e-12, max_iter=60, theta=0.5, cycle=cycle,
                 pmg=dict(tol=1e-13, precision=precision))
    assert st["levels"] == 3
    assert _rel(U, seq) < 1e-10, st


def test_forward_euler_converges_to_sequential(B):
    """Forward Euler (theta = 0: every step is a mass-matrix solve) on steps
    small enough for the coarse propagator to be stable too."""
    p, nel, T, Nt = 2, 8, 8e-4, 32
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C, theta=0.0)
    U, st = _gpu(B, p, nel, T, Nt, m=4, max_levels=2, tol=1e-12, max_iter=40, theta=0.0,
                 pmg=dict(tol=1e-13, precision=0))
    assert _rel(U, seq) < 1e-10, st


def test_curved_theta_rhs(B):
    """The explicit part of the step on the curved map (stencil path)."""
    p, nel, T, Nt = 2, 8, 0.5, 32
    d = assembly.Discretisation(p, nel, geometry.QuarterAnnulus())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C, theta=0.5)
    U, st = _gpu(B, p, nel, T, Nt, geom="quarter_annulus", m=4, tol=1e-12, max_iter=60,
                 theta=0.5, pmg=dict(tol=1e-13, precision=0))
    assert _rel(U, seq) < 1e-10, st


def test_invalid_variant_options_rejected(B):
    prob = B.Problem(2, 8)
    for bad in (dict(theta=1.5), dict(theta=-0.1), dict(cycle=3)):
        with pytest.raises(B.IgmError):
            B.MGRIT(prob, T=1.0, Nt=16, **bad)


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("geom", ["unit_square", "quarter_annulus"])
def test_cg_fixed_iterations_match_oracle(B, geom):
    """k iterations of the diagonally preconditioned CG (pmg_opts.solver = 1)
    from a random start equal the oracle's PCG iterates (several columns)."""
    from oracle import cg
    p, nel, c = 3, 16, 1.0 / 256
    d = assembly.Discretisation(p, nel, geometry.get(geom))
    A = (d.M + c * d.K).tocsr()
    rng = np.random.default_rng(11)
    b = rng.standard_normal((3, d.N))
    x0 = rng.standard_normal((3, d.N))
    prob = B.Problem(p, nel, geom)
    g = B.PMG(prob, c, solver=1, precision=1)   # CG always runs in FP64
    for k in (1, 5, 20):
        X = _cuda(x0)
        cyc, _ = g.solve(_cuda(b), X, ncycles=k, check=False)
        assert list(cyc) == [k] * 3
        for j in range(3):
            want, _ = cg.pcg_jacobi(A, b[j], x0[j], niter=k)
            assert _rel(X[j].cpu().numpy(), want) < 1e-9, (k, j)


def test_cg_converged_vs_direct_and_iterations_grow_with_p(B):
    from scipy.sparse.linalg import spsolve
    its = []
    for p in (2, 3, 4, 5):
        d = assembly.Discretisation(p, 16, geometry.UnitSquare())
        A = (d.M + d.K / 256.0).tocsc()
        b = d.load_vector(lambda xi, eta, x, y: np.ones_like(x))
        g = B.PMG(B.Problem(p, 16), 1.0 / 256, solver=1, tol=1e-12, max_cycles=5000)
        X = _cuda(np.zeros((1, d.N)))
        cyc, _ = g.solve(_cuda(b[None, :]), X)
        assert _rel(X[0].cpu().numpy(), spsolve(A, b)) < 1e-10
        its.append(int(cyc[0]))
    assert all(b > a for a, b in zip(its, its[1:])), its


def test_mgrit_with_cg_spatial_solves(B):
    """MGRIT whose every step is solved by CG reaches sequential backward Euler."""
    p, nel, T, Nt = 3, 16, 1.0, 64
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C)
    U, st = _gpu(B, p, nel, T, Nt, m=4, tol=1e-12, max_iter=60,
                 pmg=dict(solver=1, tol=1e-13, max_cycles=5000))
    assert st["levels"] == 3
    assert _rel(U, seq) < 1e-10, st
    assert st["vcyc_mean"] > 5   # CG iterations per solve, not p-multigrid cycles


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("solver", [0, 1])
def test_tiny_right_hand_side_scales_exactly(B, precision, solver):
    """A right-hand side 2^-200 times smaller (far below FP32's range, as a
    decayed solution produces) gives exactly 2^-200 times the solution: the
    solves scale by powers of two internally."""
    import torch
    d = assembly.Discretisation(3, 16, geometry.UnitSquare())
    b = np.random.default_rng(4).standard_normal((2, d.N))
    g = B.PMG(B.Problem(3, 16), 1.0 / 64, precision=precision, solver=solver, tol=1e-10,
              max_cycles=2000)
    X1 = torch.zeros((2, d.N), dtype=torch.float64, device="cuda")
    X2 = torch.zeros_like(X1)
    c1, _ = g.solve(torch.as_tensor(b, device="cuda"), X1)
    c2, _ = g.solve(torch.as_tensor(np.ldexp(b, -200), device="cuda"), X2)
    assert list(c1) == list(c2) and min(c1) > 0
    np.testing.assert_array_equal(np.ldexp(X1.cpu().numpy(), -200), X2.cpu().numpy())


def test_coarse_cycles_fixed_iterations_match_oracle(B):
    """One p-multigrid cycle per coarse-level solve (FP64 form): k MGRIT
    iterations equal the oracle's with the same inexact coarse propagator."""
    p, nel, T, Nt, m = 2, 8, 1.0, 64, 4
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    lo = assembly.Discretisation(1, nel, geometry.UnitSquare())
    u0, fhat = d.project(S), d.load_vector(S)
    for k in (1, 2):
        mg = mgrit.MGRIT(d.M, d.K, 1.0, T, Nt, m,
                         mgrit.pmg_factory(d, lo, tol=1e-14, max_cycles=60, coarse_cycles=1),
                         u0, fhat, C)
        Uo, it, hist = mg.run(tol=0.0, max_iter=k)
        U, st = _gpu(B, p, nel, T, Nt, check=False, m=m, tol=0.0, max_iter=k, coarse_cycles=1,
                     pmg=dict(tol=1e-14, precision=0, max_cycles=60))
        assert st["iters"] == k and st["levels"] == 3
        assert _rel(U, Uo) < 1e-9, k
        np.testing.assert_allclose(st["res_hist"], hist, rtol=1e-7)


@pytest.mark.parametrize("precision", [0, 1])
def test_coarse_cycles_converge_to_sequential(B, precision):
    p, nel, T, Nt = 3, 16, 1.0, 256
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S), d.load_vector(S), C)
    U, st = _gpu(B, p, nel, T, Nt, m=4, tol=1e-12, max_iter=60, coarse_cycles=1,
                 pmg=dict(tol=1e-13, precision=precision))
    assert st["levels"] == 4
    assert _rel(U, seq) < 1e-10, st


@pytest.mark.parametrize("p", [2, 5])
def test_autotuned_layout_gives_the_same_solve(B, p):
    """pmg_opts.autotune = 1 (layout chosen by timing) solves like the default
    layout: fixed FP64 cycles equal the oracle's, converged mixed solves agree."""
    import torch
    from oracle import pmg as opmg
    nel, c = 16, 1.0 / 256
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    lo = assembly.Discretisation(1, nel, geometry.UnitSquare())
    b = np.random.default_rng(8).standard_normal((2, d.N))
    P = opmg.PMG(d, lo, c)
    want = np.array([P.solve(bb, np.zeros(d.N), ncycles=2)[0] for bb in b])
    g = B.PMG(B.Problem(p, nel), c, precision=0, autotune=1)
    X = torch.zeros((2, d.N), dtype=torch.float64, device="cuda")
    g.solve(torch.as_tensor(b, device="cuda"), X, ncycles=2, check=False)
    assert _rel(X.cpu().numpy(), want) < 1e-10
    sols = []
    for tune in (0, 1):
        gm = B.PMG(B.Problem(p, nel), c, precision=1, tol=1e-12, autotune=tune)
        Y = torch.zeros((2, d.N), dtype=torch.float64, device="cuda")
        gm.solve(torch.as_tensor(b, device="cuda"), Y)
        sols.append(Y.cpu().numpy())
    assert _rel(sols[1], sols[0]) < 1e-10


@pytest.mark.parametrize("p,nel", [(2, 16), (4, 24), (5, 8)])
@pytest.mark.parametrize("which", ["M", "K", "A"])
def test_batched_fp32_operator_apply_matches_oracle(B, p, nel, which):
    """iga_apply_f32 (FP32 sum factorisation over a block of columns) against
    the oracle's assembled M, K in FP64: FP32 rounding only."""
    import torch
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    c = 0.37
    A = {"M": d.M, "K": d.K, "A": d.M + c * d.K}[which]
    X = np.random.default_rng(6).standard_normal((7, d.N))
    want = np.array([A @ x for x in X])
    prob = B.Problem(p, nel)
    Y = prob.apply_f32(which, torch.as_tensor(X, dtype=torch.float32, device="cuda"), c=c)
    got = Y.double().cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-6


@pytest.mark.parametrize("p,nel,pad", [(2, 16, 3), (3, 20, 1), (5, 12, 0), (2, 80, 5)])
def test_batched_fp32_apply_many_columns_per_cta(B, p, nel, pad):
    """Several columns per persistent CTA (ring-slot reuse, both (tm, tk)
    buffers, the buffer hand-back), a leading dimension that is not a multiple
    of four, and (nel = 80: 80 grid lines) the wider shared-memory layout;
    every column against the oracle's assembled M + c K."""
    import torch
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    c = 1.0 / 256
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nrhs = 4 * sms + 37
    X = np.random.default_rng(7).standard_normal((nrhs, d.N + pad))
    want = ((d.M + c * d.K) @ X[:, :d.N].T).T
    prob = B.Problem(p, nel)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    Y = prob.apply_f32("A", Xd, c=c)
    got = Y[:, :d.N].double().cpu().numpy()
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() < 2e-6
    assert torch.equal(Xd, torch.as_tensor(X, dtype=torch.float32, device="cuda"))


def test_batched_fp32_apply_full_size_sampled(B):
    """The measured configuration (p = 4, h = 1/64, 8192 columns padded to a
    multiple of four floats, one launch): sampled columns, including the first
    and last of a CTA's share, against the oracle."""
    import torch
    p, nel, ncol = 4, 64, 8192
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    c = 1.0 / 256
    ld = (d.N + 3) // 4 * 4
    g = torch.Generator(device="cuda").manual_seed(11)
    Xd = torch.randn((ncol, ld), dtype=torch.float32, device="cuda", generator=g)
    Y = B.Problem(p, nel).apply_f32("A", Xd, c=c)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cols = sorted({0, 1, sms - 1, sms, 2 * sms + 5, ncol // 2, ncol - sms, ncol - 1}
                  | set(np.random.default_rng(8).integers(0, ncol, 16).tolist()))
    X = Xd[cols, :d.N].double().cpu().numpy()
    want = ((d.M + c * d.K) @ X.T).T
    got = Y[cols, :d.N].double().cpu().numpy()
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() < 2e-6


@pytest.mark.parametrize("p,nel", [(2, 1024), (3, 512)])
def test_batched_fp32_apply_row_strips_largest_grid(B, p, nel):
    """The largest grid a descriptor allows (1024 x 1024 elements, n = 1024 grid
    lines) and n = 513 at p = 3: more grid columns than a CTA has threads, so
    threads walk two of them (at n = 513 one thread alone takes the second).
    Sampled outputs at the edges, the corners,
    the strip boundaries and the thread-chunk boundary, against stencil rows
    taken from the oracle's small problem by translation and scaling."""
    import torch
    nel_s, ncol = 4 * p + 2, 3
    ds = assembly.Discretisation(p, nel_s, geometry.UnitSquare())
    prob = B.Problem(p, nel)
    n = prob.n
    c = 1.0 / 4096
    g = torch.Generator(device="cuda").manual_seed(15)
    Xd = torch.randn((ncol, prob.N), dtype=torch.float32, device="cuda", generator=g)
    Y = prob.apply_f32("A", Xd, c=c).double().cpu().numpy().reshape(ncol, n, n)
    X = Xd.double().cpu().numpy().reshape(ncol, n, n)
    rng = np.random.default_rng(16)
    pts = {(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (31, 511), (32, 512),
           (n // 2, 1), (2, n - 3), (n - 2 * p, 2 * p - 1), (63, n - 1), (64, 0)}
    pts |= {tuple(v) for v in rng.integers(0, n, (24, 2)).tolist()}
    got, want = [], []
    for iy, ix in sorted(pts):
        st = unit_square_row(ds, nel_s, nel, p, n, iy, ix)
        for b in range(ncol):
            w = sum((m + c * k) * X[b, iy + dy, ix + dx] for (dy, dx), (m, k) in st.items())
            got.append(Y[b, iy, ix])
            want.append(w)
    got, want = np.array(got), np.array(want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-6


def _curved_bound(d, which, c, X32):
    """Elementwise bound on the FP32 apply of an assembled stencil (Sec. 2, M and
    K on the curved map): each coefficient a = fl(cm M + ck K) is within
    3u (|M| + |c| |K|) of the exact value (rounding of M, K, c and of the
    FMA), and the Q-term FMA chain adds at most gamma_Q < (Q + 1) u of
    sum |a_i x_i| (u = 2^-24, Q = (2p+1)^2; x is taken as its FP32 value)."""
    absM, absK = abs(d.M), abs(d.K)
    mag = {"M": absM, "K": absK, "A": absM + abs(c) * absK}[which]
    Q = (2 * d.p + 1) ** 2
    return (Q + 4) * 2.0 ** -24 * (mag @ np.abs(X32).T).T


@pytest.mark.parametrize("p,nel,nrhs,pad", [(2, 40, 7, 0), (3, 64, 101, 3), (4, 36, 13, 1),
                                            (5, 12, 250, 2), (6, 10, 9, 0)])
@pytest.mark.parametrize("which", ["M", "K", "A"])
def test_batched_fp32_apply_curved_map(B, p, nel, nrhs, pad, which):
    """The curved-map form of iga_apply_f32 on the quarter annulus against the
    oracle's assembled M, K (FP64) on the same FP32 inputs, element by element
    within the rounding bound of the arithmetic: ragged 8 x 32 tiles (n = 40,
    38, 15), a column count that is not a multiple of four, several column
    groups per CTA (n = 65, 101 columns), a padded leading dimension, and
    p = 6 (coefficients read from global memory instead of registers)."""
    import torch
    d = assembly.Discretisation(p, nel, geometry.QuarterAnnulus())
    c = 0.37
    A = {"M": d.M, "K": d.K, "A": d.M + c * d.K}[which]
    X = np.random.default_rng(12).standard_normal((nrhs, d.N + pad))
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    X32 = Xd[:, :d.N].double().cpu().numpy()
    want = (A @ X32.T).T
    prob = B.Problem(p, nel, "quarter_annulus")
    Y = prob.apply_f32(which, Xd, c=c)
    got = Y[:, :d.N].double().cpu().numpy()
    bound = _curved_bound(d, which, c, X32)
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)
    assert torch.equal(Xd, torch.as_tensor(X, dtype=torch.float32, device="cuda"))


def test_batched_fp32_apply_curved_full_size_sampled(B):
    """The annulus_c3 grid (p = 4, 128 x 128 elements, n = 130) with 1024 columns
    in one launch: sampled columns, including the first and last, against the
    oracle's assembled M + c K within the rounding bound."""
    import torch
    p, nel, ncol = 4, 128, 1024
    d = assembly.Discretisation(p, nel, geometry.QuarterAnnulus())
    c = 1.0 / 1024
    g = torch.Generator(device="cuda").manual_seed(13)
    Xd = torch.randn((ncol, d.N), dtype=torch.float32, device="cuda", generator=g)
    Y = B.Problem(p, nel, "quarter_annulus").apply_f32("A", Xd, c=c)
    cols = sorted({0, 1, 3, 4, ncol // 2, ncol - 1}
                  | set(np.random.default_rng(14).integers(0, ncol, 10).tolist()))
    X32 = Xd[cols].double().cpu().numpy()
    want = ((d.M + c * d.K) @ X32.T).T
    got = Y[cols].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= _curved_bound(d, "A", c, X32))


@pytest.mark.parametrize("geom,p,nel", [("unit_square", 4, 64), ("quarter_annulus", 3, 16)])
def test_mixed_form_with_fp64_w_cycle(B, geom, p, nel):
    """pmg_opts.hmg_fp64: the mixed form with the whole p = 1 W-cycle in FP64
    (Sec. 4, step 3; the transfers stay FP32).  One refinement step equals the
    oracle's FP64 cycle to FP32 rounding, converged solves equal the direct
    solution to 1e-10, and an MGRIT run equals sequential stepping."""
    import scipy.sparse as sp
    import torch
    from scipy.sparse.linalg import splu
    from oracle import pmg as opmg
    from paper_2107_05337_gb300 import inputs
    _cuda = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    c = 1.0 / 256
    prob = B.Problem(p, nel, geom)
    hi, lo = assembly.problem(p, nel, geometry.get(geom))
    P = opmg.PMG(hi, lo, c)
    g = B.PMG(prob, c, precision=1, tol=1e-12, hmg_fp64=1)
    Bm = inputs.random_block(71, prob.N, 2)
    X = _cuda(np.zeros_like(Bm))
    g.solve(_cuda(Bm), X, ncycles=1)
    X = X.cpu().numpy()
    for k in range(2):
        x, _ = P.solve(Bm[k], np.zeros(prob.N), ncycles=1)
        assert _rel(X[k], x) < 2e-5, k
    X = _cuda(np.zeros_like(Bm))
    g.solve(_cuda(Bm), X)
    X = X.cpu().numpy()
    lu = splu(sp.csc_matrix(P.A))
    for k in range(2):
        assert _rel(X[k], lu.solve(Bm[k])) < 1e-10, k
    if geom == "unit_square":
        d = assembly.Discretisation(p, 16, geometry.UnitSquare())
        seq = timestep.sequential(d.M, d.K, 1.0, 1.0, 64, d.project(S), d.load_vector(S), C)
        U, st = _gpu(B, p, 16, 1.0, 64, m=4, tol=1e-12,
                     pmg=dict(tol=1e-13, precision=1, hmg_fp64=1))
        assert _rel(U, seq) < 1e-10, st


@pytest.mark.parametrize("p,nel,nrhs", [(5, 128, 5), (2, 100, 700), (3, 90, 9)])
def test_batched_fp32_apply_row_strips_beyond_84_lines(B, p, nel, nrhs):
    """Grids the persistent layouts do not hold (n = nel + p - 2 > 84: the
    h = 1/128 grids of batch_c5) go through the row-strip form; every column
    against the oracle's assembled M + c K (Sec. 2, Eq. (los)), a ragged last
    strip, and (700 columns) several columns per CTA through both copy stages."""
    import torch
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    assert d.n > 84
    c = 1.0 / 512
    X = np.random.default_rng(9).standard_normal((nrhs, d.N))
    want = ((d.M + c * d.K) @ X.T).T
    prob = B.Problem(p, nel)
    Y = prob.apply_f32("A", torch.as_tensor(X, dtype=torch.float32, device="cuda"), c=c)
    got = Y.double().cpu().numpy()
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() < 2e-6, err
    for which, A in (("M", d.M), ("K", d.K)):
        Y = prob.apply_f32(which, torch.as_tensor(X[:2], dtype=torch.float32, device="cuda"))
        w = (A @ X[:2].T).T
        assert np.linalg.norm(Y.double().cpu().numpy() - w) / np.linalg.norm(w) < 2e-6, which
