"""Learned coarse propagator for MGRIT and the FAS two-level cycle that uses
it, plain FP64 (numpy).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_learned.py``:
  * the back-propagated gradients (weights and network input) equal central
    finite differences of the loss;
  * GELU and its derivative against the closed form at known points and
    against finite differences;
  * Phi_c(0) = 0 and Phi_c(a u) = a Phi_c(u) for a > 0 (the input is
    normalised by its maximum modulus); with the last layer zero Phi_c is the
    identity;
  * a network whose kernels are all the centre tap reduces to a pointwise
    composition of GELUs (checked against the scalar formula);
  * FAS two-level MGRIT with Phi_c = the backward-Euler coarse propagator
    reproduces the correction-scheme two-level iterates (the coarse equations
    coincide for a linear Phi_c);
  * for any Phi_c (random weights) the FAS fixed point is sequential stepping,
    because the fine propagator is unchanged (Sec. 3: the fixed point is the
    block forward solve of A u = g);
  * a propagator that does not contract (here -identity) is replaced by the
    backward-Euler one once the residual contraction after a learned
    correction exceeds 0.5; that correction is undone first.

The network (reading; the paper uses only the rediscretised coarse step): on
the n x n grid of interior coefficients (zero padding = the homogeneous
Dirichlet condition), x = u / s with s = max |u|,
    h1 = g(K1 * x),  h2 = g(K2 * h1),  h3 = g(K3 * h2),
    Phi_c(u) = s (x + K4 * h3),
four 3 x 3 convolutions K1 (1 -> C), K2, K3 (C -> C), K4 (C -> 1) with C = 32
channels, no biases (so Phi_c(0) = 0 and Phi_c is positively homogeneous), and
the GELU g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (Phi the standard
normal distribution function).  Trained on pairs (u_n, u_{n+m}) of the fine
stepper by the mean squared error of Phi_c(u_n)/s - u_{n+m}/s, Adam.

FAS two-level cycle (two levels, m fine steps per coarse step, coarse unknowns
v_j at the C-points t_{jm}): after FCF relaxation of the fine level, with the
C-point residuals r_j = Phi(u_{jm-1}) + g_{jm} - u_{jm},
    tau_j = u_{jm} - Phi_c(u_{(j-1)m}) + r_j,
    v_0 = u_0,  v_j = Phi_c(v_{j-1}) + tau_j  (sequential),
    u_{jm} <- v_j, then F-relaxation (ideal interpolation).
If the residual after a learned correction is not finite or contracted by
more than the switch ratio (0.5), the iterate before the correction is
restored and relaxed again, and the backward-Euler coarse propagator is used
from then on.
"""
import math

import numpy as np
from scipy.special import erf

KS = 3  # kernel size
LAYERS = 4


def gelu(z):
    """z Phi(z) with Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_deriv(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def conv2d(x, w):
    """'Same' convolution with zero padding: x [Cin, n, n], w [Cout, Cin, KS, KS]
    -> [Cout, n, n]; out[o,i,j] = sum_{c,a,b} w[o,c,a,b] x[c, i+a-h, j+b-h],
    h = KS // 2."""
    cin, n, _ = x.shape
    h = KS // 2
    xp = np.zeros((cin, n + 2 * h, n + 2 * h))
    xp[:, h:h + n, h:h + n] = x
    out = np.zeros((w.shape[0], n, n))
    for a in range(KS):
        for b in range(KS):
            out += np.einsum("oc,cij->oij", w[:, :, a, b], xp[:, a:a + n, b:b + n])
    return out


def conv2d_grads(x, w, gout):
    """Gradients of sum(gout * conv2d(x, w)) with respect to x and w."""
    cin, n, _ = x.shape
    h = KS // 2
    xp = np.zeros((cin, n + 2 * h, n + 2 * h))
    xp[:, h:h + n, h:h + n] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for a in range(KS):
        for b in range(KS):
            gw[:, :, a, b] = np.einsum("oij,cij->oc", gout, xp[:, a:a + n, b:b + n])
            gxp[:, a:a + n, b:b + n] += np.einsum("oc,oij->cij", w[:, :, a, b], gout)
    return gxp[:, h:h + n, h:h + n], gw


class ConvNet:
    def __init__(self, n, channels=32, seed=0, zero_last=True):
        rng = np.random.default_rng(seed)
        c = channels
        self.n = n
        self.C = c
        self.W = [rng.standard_normal((c, 1, KS, KS)) / KS,
                  rng.standard_normal((c, c, KS, KS)) / (KS * np.sqrt(c)),
                  rng.standard_normal((c, c, KS, KS)) / (KS * np.sqrt(c)),
                  np.zeros((1, c, KS, KS)) if zero_last else
                  rng.standard_normal((1, c, KS, KS)) / (KS * np.sqrt(c))]

    def forward_normalised(self, x, keep=False):
        """x [n, n] (already normalised) -> network output [n, n]."""
        a = [x[None]]
        zs = []
        for k in range(LAYERS - 1):
            z = conv2d(a[-1], self.W[k])
            zs.append(z)
            a.append(gelu(z))
        y = x + conv2d(a[-1], self.W[LAYERS - 1])[0]
        if keep:
            return y, (a, zs)
        return y

    def __call__(self, u):
        """Phi_c on a coefficient vector u [n*n] (xi fastest)."""
        s = np.abs(u).max()
        if s == 0.0:
            return np.zeros_like(u)
        x = (u / s).reshape(self.n, self.n)
        return s * self.forward_normalised(x).ravel()

    def loss_and_grads(self, X, Y, input_grad=False):
        """Mean squared error over a batch of normalised pairs X, Y [B, n, n] and
        its gradient with respect to the four kernels (and, with input_grad,
        with respect to every input X_b, as [B, n, n])."""
        G = [np.zeros_like(w) for w in self.W]
        GX = np.zeros_like(X)
        loss = 0.0
        B = X.shape[0]
        npix = self.n * self.n
        for b, (x, yt) in enumerate(zip(X, Y)):
            y, (a, zs) = self.forward_normalised(x, keep=True)
            d = y - yt
            loss += float(np.sum(d * d)) / (B * npix)
            gy = (2.0 / (B * npix)) * d
            gin, gw = conv2d_grads(a[LAYERS - 1], self.W[LAYERS - 1], gy[None])
            G[LAYERS - 1] += gw
            for k in range(LAYERS - 2, -1, -1):
                gz = gin * gelu_deriv(zs[k])
                gin, gw = conv2d_grads(a[k], self.W[k], gz)
                G[k] += gw
            GX[b] = gy + gin[0]          # the skip connection and the network
        if input_grad:
            return loss, G, GX
        return loss, G


def normalised_pairs(U0, U1, n):
    """(u_n, u_{n+m}) rows -> normalised [B, n, n] inputs and targets (scale of
    each input; rows with u_n = 0 are dropped)."""
    s = np.abs(U0).max(axis=1)
    keep = s > 0
    X = (U0[keep] / s[keep, None]).reshape(-1, n, n)
    Y = (U1[keep] / s[keep, None]).reshape(-1, n, n)
    return X, Y


def train(net, X, Y, steps, batch=16, lr=1e-3, seed=0, b1=0.9, b2=0.999, eps=1e-8):
    """Adam on the mean squared error; returns the loss history."""
    rng = np.random.default_rng(seed)
    m = [np.zeros_like(w) for w in net.W]
    v = [np.zeros_like(w) for w in net.W]
    hist = []
    for t in range(1, steps + 1):
        idx = rng.integers(0, X.shape[0], size=min(batch, X.shape[0]))
        loss, G = net.loss_and_grads(X[idx], Y[idx])
        hist.append(loss)
        for k in range(len(net.W)):
            m[k] = b1 * m[k] + (1 - b1) * G[k]
            v[k] = b2 * v[k] + (1 - b2) * G[k] * G[k]
            mh = m[k] / (1 - b1 ** t)
            vh = v[k] / (1 - b2 ** t)
            net.W[k] = net.W[k] - lr * mh / (np.sqrt(vh) + eps)
    return hist


class FASTwoLevel:
    """Two-level MGRIT, FCF relaxation, FAS coarse equation with a (possibly
    nonlinear) coarse propagator phi_c; falls back to fallback_c when the
    residual contraction rho_k / rho_{k-1} exceeds `switch` (0.5).

    step(u, n) -> Phi(u) + g_n for the fine step into point n; u0 the initial value."""

    def __init__(self, step, phi_c, fallback_c, u0, Nt, m, switch=0.5):
        self.step, self.phi_c, self.fallback_c = step, phi_c, fallback_c
        self.Nt, self.m, self.switch = Nt, m, switch
        self.U = np.zeros((Nt + 1, len(u0)))
        self.U[0] = u0
        self.used_fallback = False

    def _f_relax(self):
        for j in range(self.Nt // self.m):
            for k in range(1, self.m):
                n = j * self.m + k
                self.U[n] = self.step(self.U[n - 1], n)

    def _c_relax(self):
        for j in range(1, self.Nt // self.m + 1):
            n = j * self.m
            self.U[n] = self.step(self.U[n - 1], n)

    def run(self, tol=1e-10, max_iter=50):
        m, Nc = self.m, self.Nt // self.m
        hist = []
        phic = self.phi_c
        it = 0
        backup = None
        while True:
            if it == 0:
                self._f_relax()
            self._c_relax()
            self._f_relax()
            r = [self.step(self.U[j * m - 1], j * m) - self.U[j * m] for j in range(1, Nc + 1)]
            rho = np.sqrt(sum(float(x @ x) for x in r))
            if backup is not None and not (rho <= self.switch * hist[-1]):
                # the learned correction is undone; backward Euler from here on
                self.U = backup
                backup = None
                phic = self.fallback_c
                self.used_fallback = True
                continue
            backup = None
            hist.append(rho)
            if rho == 0.0 or rho <= tol * hist[0] or it >= max_iter:
                break
            if phic is not self.fallback_c:
                backup = self.U.copy()
            C = [self.U[j * m].copy() for j in range(Nc + 1)]
            tau = [None] + [C[j] - phic(C[j - 1]) + r[j - 1] for j in range(1, Nc + 1)]
            v = C[0].copy()
            for j in range(1, Nc + 1):
                v = phic(v) + tau[j]
                self.U[j * m] = v
            self._f_relax()
            it += 1
        return self.U, it, hist
