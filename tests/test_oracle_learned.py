"""Pins of the oracle's learned coarse propagator and FAS two-level MGRIT."""
import numpy as np
from scipy.sparse.linalg import splu

from oracle import assembly, geometry, learned, mgrit, timestep

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y) + 0.3 * np.sin(3 * np.pi * x) * np.sin(2 * np.pi * y)


def test_gradient_matches_finite_differences():
    """Back-propagation through the four 3 x 3 layers and three GELUs: the
    weight gradients of every layer and the gradient with respect to the
    network input equal central differences of the loss."""
    n = 7
    net = learned.ConvNet(n, channels=2, seed=3, zero_last=False)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((2, n, n))
    Y = rng.standard_normal((2, n, n))
    _, G, GX = net.loss_and_grads(X, Y, input_grad=True)
    h = 1e-6
    for k, idx in ((0, (1, 0, 2, 1)), (1, (0, 1, 0, 0)), (2, (1, 0, 1, 2)), (3, (0, 1, 2, 2)),
                   (1, (1, 1, 1, 1)), (3, (0, 0, 0, 1))):
        w0 = net.W[k][idx]
        net.W[k][idx] = w0 + h
        lp, _ = net.loss_and_grads(X, Y)
        net.W[k][idx] = w0 - h
        lm, _ = net.loss_and_grads(X, Y)
        net.W[k][idx] = w0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[k][idx]) <= 1e-7 * max(1.0, abs(fd)), (k, idx, fd, G[k][idx])
    for idx in ((0, 3, 3), (1, 0, 6), (1, 4, 2)):
        x0 = X[idx]
        X[idx] = x0 + h
        lp, _ = net.loss_and_grads(X, Y)
        X[idx] = x0 - h
        lm, _ = net.loss_and_grads(X, Y)
        X[idx] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - GX[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, GX[idx])


def test_gelu_closed_form_and_derivative():
    """g(z) = z Phi(z): g(0) = 0, g(1) = Phi(1), g(-1) = -(1 - Phi(1)) with the
    tabulated Phi(1) = 0.8413447460685429; g(z) -> z and g(-z) -> 0 for large
    z; g'(0) = 1/2 and g' against central differences."""
    phi1 = 0.8413447460685429
    z = np.array([0.0, 1.0, -1.0, 8.0, -8.0])
    np.testing.assert_allclose(learned.gelu(z), [0.0, phi1, -(1.0 - phi1), 8.0, 0.0],
                               rtol=1e-14, atol=1e-13)
    assert learned.gelu_deriv(np.array(0.0)) == 0.5
    zz = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (learned.gelu(zz + h) - learned.gelu(zz - h)) / (2 * h)
    np.testing.assert_allclose(learned.gelu_deriv(zz), fd, rtol=0, atol=1e-8)


def test_centre_tap_network_is_pointwise():
    """With every kernel zero except its centre tap and one channel, the
    convolutions are pointwise products and Phi_c(u)/s = x + w4 g(w3 g(w2
    g(w1 x))) at every grid point."""
    n = 5
    net = learned.ConvNet(n, channels=1, seed=0, zero_last=False)
    w = [0.7, -1.3, 0.9, 1.1]
    for k in range(4):
        net.W[k][:] = 0.0
        net.W[k][0, 0, 1, 1] = w[k]
    x = np.random.default_rng(5).uniform(-1, 1, (n, n))
    want = x + w[3] * learned.gelu(w[2] * learned.gelu(w[1] * learned.gelu(w[0] * x)))
    np.testing.assert_allclose(net.forward_normalised(x), want, rtol=1e-15, atol=1e-15)


def test_zero_homogeneity_and_identity_start():
    n = 9
    net = learned.ConvNet(n, channels=3, seed=1, zero_last=False)
    u = np.random.default_rng(2).standard_normal(n * n)
    assert np.all(net(np.zeros(n * n)) == 0.0)
    np.testing.assert_allclose(net(4.0 * u), 4.0 * net(u), rtol=1e-14, atol=1e-14)
    ident = learned.ConvNet(n, channels=3, seed=1, zero_last=True)
    np.testing.assert_allclose(ident(u), u, rtol=0, atol=1e-15)


def _problem(nel=6, p=2, Nt=32, m=4, T=0.5):
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    dt = T / Nt
    fine = splu((d.M + dt * d.K).tocsc())
    coarse = splu((d.M + m * dt * d.K).tocsc())
    step = lambda u, n: fine.solve(d.M @ u)
    be_c = lambda u: coarse.solve(d.M @ u)
    return d, step, be_c


def test_fas_with_linear_coarse_propagator_equals_correction_scheme():
    d, step, be_c = _problem()
    u0 = d.project(S)
    for k in (1, 2, 3):
        fas = learned.FASTwoLevel(step, be_c, be_c, u0, 32, 4)
        Uf, itf, hf = fas.run(tol=0.0, max_iter=k)
        cs = mgrit.MGRIT(d.M, d.K, 1.0, 0.5, 32, 4, mgrit.direct_factory(d.M, d.K), u0,
                         max_levels=2)
        Uc, itc, hc = cs.run(tol=0.0, max_iter=k)
        assert itf == itc == k
        np.testing.assert_allclose(Uf, Uc, rtol=0, atol=1e-13 * np.abs(Uc).max())
        np.testing.assert_allclose(hf, hc, rtol=1e-10)


def test_fas_fixed_point_is_sequential_for_any_propagator():
    d, step, be_c = _problem()
    u0 = d.project(S)
    seq = timestep.sequential(d.M, d.K, 1.0, 0.5, 32, u0)
    net = learned.ConvNet(d.n, channels=2, seed=7, zero_last=False)
    fas = learned.FASTwoLevel(step, net, be_c, u0, 32, 4, switch=2.0)   # never fall back
    U, it, hist = fas.run(tol=1e-13, max_iter=60)
    assert not fas.used_fallback
    np.testing.assert_allclose(U, seq, rtol=0, atol=1e-12 * np.abs(seq).max())


def test_non_contracting_propagator_falls_back():
    d, step, be_c = _problem()
    u0 = d.project(S)
    seq = timestep.sequential(d.M, d.K, 1.0, 0.5, 32, u0)
    bad = lambda u: -u
    fas = learned.FASTwoLevel(step, bad, be_c, u0, 32, 4)
    U, it, hist = fas.run(tol=1e-12, max_iter=40)
    assert fas.used_fallback
    np.testing.assert_allclose(U, seq, rtol=0, atol=1e-10 * np.abs(seq).max())


def test_training_fits_the_coarse_step():
    """Trained on pairs (u, BE_c(u)) of the coarse backward-Euler step, the
    network's error falls well below the identity's."""
    d, step, be_c = _problem(nel=6, p=2)
    rng = np.random.default_rng(0)
    U0 = rng.standard_normal((24, d.N))
    # smooth inputs: a few applications of the step
    for _ in range(2):
        U0 = np.array([be_c(u) for u in U0])
    U1 = np.array([be_c(u) for u in U0])
    X, Y = learned.normalised_pairs(U0, U1, d.n)
    net = learned.ConvNet(d.n, channels=4, seed=0)
    e0 = np.mean((X - Y) ** 2)
    hist = learned.train(net, X, Y, steps=150, batch=8, lr=3e-3)
    assert hist[-1] < 0.25 * e0, (e0, hist[-1])
