"""GPU: the learned coarse propagator (BF16 network kernels, the C -> C
layers on the tensor cores) against the oracle network, its gradients and
training, and two-level FAS MGRIT with it."""
import numpy as np
import pytest

from oracle import assembly, geometry, learned, timestep

pytestmark = pytest.mark.gpu

S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y) + 0.3 * np.sin(3 * np.pi * x) * np.sin(2 * np.pi * y)


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_05337_gb300 import binding
    binding.lib()
    return binding


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _flat(net):
    return np.concatenate([w.ravel() for w in net.W]).astype(np.float32)


def _fp32_weights(net):
    # weights exactly representable in FP32, as the GPU holds them
    for k in range(len(net.W)):
        net.W[k] = net.W[k].astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,C", [(12, 16), (23, 32)])
def test_forward_matches_oracle(B, n, C):
    """Same weights: the GPU network's correction Phi_c(u) - u equals the
    oracle's to BF16 accuracy (several random inputs, one of them tiny: the
    input normalisation)."""
    net = learned.ConvNet(n, channels=C, seed=5, zero_last=False)
    _fp32_weights(net)
    g = B.Phic(n, C)
    g.weights = _flat(net)
    np.testing.assert_array_equal(g.weights, _flat(net))
    U = np.random.default_rng(1).standard_normal((3, n * n)) * np.array([[1.0], [1e-30], [7.5]])
    out = g.apply(_cuda(U)).cpu().numpy()
    for b in range(3):
        want = net(U[b])
        corr_g, corr_o = out[b] - U[b], want - U[b]
        assert np.linalg.norm(corr_g - corr_o) <= 3e-2 * np.linalg.norm(corr_o), b
    assert np.all(g.apply(_cuda(np.zeros((1, n * n)))).cpu().numpy() == 0.0)


def _close(got, want, what):
    """BF16 tolerance: activations, pre-activations and the back-propagated
    gradients are rounded to 8 significant bits at every layer (relative
    rounding 2^-9 each, about a dozen roundings on any path), so entries agree
    to 4e-2 of the largest entry of their tensor plus 4e-2 of themselves, and
    the tensor to 3e-2 in norm."""
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    scale = np.abs(want).max()
    assert np.all(np.abs(got - want) <= 4e-2 * scale + 4e-2 * np.abs(want)), what
    assert np.linalg.norm(got - want) <= 3e-2 * np.linalg.norm(want), what


@pytest.mark.parametrize("n,C,nb", [(10, 16, 3), (19, 32, 2)])
def test_gradients_match_oracle_elementwise(B, n, C, nb):
    """The back-propagation kernels (tensor-core input and weight gradients of
    the C -> C layers, the FMA kernels of the one-channel layers) against the
    oracle's finite-difference-pinned gradients, element by element: the loss,
    the gradient of every kernel, and the gradient with respect to the
    normalised inputs."""
    net = learned.ConvNet(n, channels=C, seed=2, zero_last=False)
    _fp32_weights(net)
    rng = np.random.default_rng(3)
    U0 = rng.standard_normal((nb, n * n))
    U1 = 0.8 * U0 + 0.1 * rng.standard_normal((nb, n * n))
    X, Y = learned.normalised_pairs(U0, U1, n)
    loss_o, G, GX = net.loss_and_grads(X, Y, input_grad=True)
    g = B.Phic(n, C)
    g.weights = _flat(net)
    loss, gw, gx = g.grad(_cuda(U0), _cuda(U1))
    assert abs(loss - loss_o) <= 2e-2 * loss_o, (loss, loss_o)
    off = 0
    for k, Gk in enumerate(G):
        _close(gw[off:off + Gk.size], Gk.ravel(), f"kernel {k + 1}")
        off += Gk.size
    assert off == gw.size
    _close(gx, GX.reshape(nb, -1), "input")


def test_adam_step_follows_the_gradient(B):
    """One training step on a single pair from fresh moments is Adam's first
    step w -= lr g / (|g| + eps) (bias-corrected moments g and g^2), with g the
    gradient phic_grad returns for the same pair and weights."""
    n, C = 10, 16
    net = learned.ConvNet(n, channels=C, seed=4, zero_last=False)
    _fp32_weights(net)
    rng = np.random.default_rng(6)
    u0 = rng.standard_normal(n * n)
    u1 = 0.7 * u0 + 0.2 * rng.standard_normal(n * n)
    g = B.Phic(n, C)
    w0 = _flat(net)
    g.weights = w0
    _, gw, _ = g.grad(_cuda(u0[None]), _cuda(u1[None]), input_grad=False)
    lr = 1e-3
    g.train(_cuda(u0[None]), _cuda(u1[None]), steps=1, batch=1, lr=lr)
    dw = g.weights.astype(np.float64) - w0
    want = -lr * gw / (np.abs(gw) + 1e-8)
    np.testing.assert_allclose(dw, want, rtol=1e-3, atol=1e-7)


def _be_pairs(d, m_dt, count=48, seed=0):
    from scipy.sparse.linalg import splu
    lu = splu((d.M + m_dt * d.K).tocsc())
    U0 = np.random.default_rng(seed).standard_normal((count, d.N))
    for _ in range(2):
        U0 = np.array([lu.solve(d.M @ u) for u in U0])
    U1 = np.array([lu.solve(d.M @ u) for u in U0])
    return U0, U1


def test_training_reduces_loss(B):
    d = assembly.Discretisation(2, 10, geometry.UnitSquare())
    U0, U1 = _be_pairs(d, 0.02)
    g = B.Phic(d.n, 16, seed=1)
    loss = g.train(_cuda(U0), _cuda(U1), steps=400, batch=16, lr=3e-3, seed=4)
    assert np.mean(loss[-20:]) < 0.2 * np.mean(loss[:5]), (loss[:5], loss[-20:])


def _trajectory(B, p, nel, T, Nt, u0fn):
    prob = B.Problem(p, nel)
    u0 = prob.project(u0fn)
    U, st, _ = B.mgrit_solve(prob, u0, T=T, Nt=Nt, max_levels=1, pmg=dict(tol=1e-13, precision=0))
    return prob, u0, U


@pytest.mark.parametrize("graphs", [1, 0])
def test_fas_mgrit_with_trained_propagator_is_sequential(B, graphs):
    """Two-level FAS MGRIT whose coarse level is the trained network converges
    to sequential backward Euler (the fine propagator is unchanged)."""
    p, nel, T, Nt, m = 2, 16, 0.5, 128, 8
    prob, u0, Useq = _trajectory(B, p, nel, T, Nt, S)
    # training pairs from the fine stepper: (u_n, u_{n+m})
    g = B.Phic(prob.n, 16, seed=3)
    loss = g.train(Useq[:-m].contiguous(), Useq[m:].contiguous(), steps=300, batch=16, lr=3e-3)
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S))
    mg = B.MGRIT(prob, T=T, Nt=Nt, m=m, max_levels=2, tol=1e-12, max_iter=60, graphs=graphs,
                 pmg=dict(tol=1e-13, precision=0))
    mg.set_coarse_propagator(g, 0.5)
    U, st, _ = mg.run(u0)
    assert np.linalg.norm(U.cpu().numpy() - seq) / np.linalg.norm(seq) < 1e-10, st
    be = B.MGRIT(prob, T=T, Nt=Nt, m=m, max_levels=2, tol=1e-12, max_iter=60,
                 pmg=dict(tol=1e-13, precision=0))
    _, st_be, _ = be.run(u0)
    assert st["iters"] <= st_be["iters"] + 3, (st["iters"], st_be["iters"], st["coarse_fallback"])


def test_non_contracting_propagator_falls_back(B):
    p, nel, T, Nt, m = 2, 8, 0.5, 64, 8
    prob = B.Problem(p, nel)
    u0 = prob.project(S)
    g = B.Phic(prob.n, 16, seed=9)
    w = g.weights
    w[-144:] = 5.0 * np.random.default_rng(0).standard_normal(144).astype(np.float32)  # K4
    g.weights = w
    d = assembly.Discretisation(p, nel, geometry.UnitSquare())
    seq = timestep.sequential(d.M, d.K, 1.0, T, Nt, d.project(S))
    mg = B.MGRIT(prob, T=T, Nt=Nt, m=m, max_levels=2, tol=1e-12, max_iter=80,
                 pmg=dict(tol=1e-13, precision=0))
    mg.set_coarse_propagator(g, 0.5)
    U, st, _ = mg.run(u0)
    assert st["coarse_fallback"] == 1
    assert np.linalg.norm(U.cpu().numpy() - seq) / np.linalg.norm(seq) < 1e-10


def test_set_propagator_needs_two_levels(B):
    prob = B.Problem(2, 8)
    g = B.Phic(prob.n, 16)
    mg = B.MGRIT(prob, T=0.5, Nt=64, m=4)   # three levels
    with pytest.raises(B.IgmError):
        mg.set_coarse_propagator(g)
