"""Sequential theta-scheme time stepping with a sparse direct spatial solve
(Sec. 2-3).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_timestep.py``:
  * on a generalised eigenvector K v = mu M v the scheme gives exactly
    u_n = ((1 - (1-theta) kappa dt mu) / (1 + theta kappa dt mu))^n v
    (backward Euler theta = 1, Crank-Nicolson 1/2, forward Euler 0);
  * the step matches a dense numpy.linalg.solve on a tiny case;
  * the manufactured solution u = sin(pi x) sin(pi y) cos t is approached at
    first order in dt (backward Euler);
  * against the exact solution of the semi-discrete system M u' + kappa K u =
    c(t) fhat (eigen-decomposition, quadrature of the source term), the error
    falls at first order for theta = 1 and at second order for theta = 1/2.

The scheme (Sec. 2, Eq. (los); Sec. 3 with general theta):
    (M + theta kappa dt K) u^{k+1} = (M - (1-theta) kappa dt K) u^k + dt f^{k+theta},
    k = 0 .. N_t-1, which is the block forward solve of the space-time system
A u = g of Sec. 3.  Reading: with a time-dependent separable source
f = c(t) fhat(x) the source term is dt (theta c(t_{k+1}) + (1-theta) c(t_k)) fhat
(for backward Euler: the source at the new time level).
"""
import numpy as np
from scipy.sparse.linalg import splu


class ThetaScheme:
    """One step (M + theta kappa dt K) u' = (M - (1-theta) kappa dt K) u + dt f."""

    def __init__(self, M, K, kappa, dt, theta=1.0):
        self.M = M.tocsr()
        self.K = K.tocsr()
        self.kappa = kappa
        self.dt = dt
        self.theta = theta
        self.A = (self.M + theta * kappa * dt * self.K).tocsc()
        self.lu = splu(self.A)

    def step(self, u, fvec=None):
        rhs = self.M @ u
        if self.theta != 1.0:
            rhs = rhs - (1.0 - self.theta) * self.kappa * self.dt * (self.K @ u)
        if fvec is not None:
            rhs = rhs + self.dt * fvec
        return self.lu.solve(rhs)


def BackwardEuler(M, K, kappa, dt):
    return ThetaScheme(M, K, kappa, dt, 1.0)


def sequential(M, K, kappa, T, Nt, u0, fhat=None, fcoef=None, theta=1.0):
    """All time levels u_0..u_Nt of sequential theta-scheme stepping, shape
    (Nt+1, N).  fcoef: callable t -> c(t), or an array of length Nt+1 (c at t_n)."""
    dt = T / Nt
    sc = ThetaScheme(M, K, kappa, dt, theta)
    U = np.zeros((Nt + 1, len(u0)))
    U[0] = u0
    for n in range(1, Nt + 1):
        fvec = None
        if fhat is not None:
            c = (lambda k: fcoef(k * dt)) if callable(fcoef) else (lambda k: fcoef[k])
            fvec = (theta * c(n) + (1.0 - theta) * c(n - 1)) * fhat
        U[n] = sc.step(U[n - 1], fvec)
    return U
