"""Sequential backward Euler with a sparse direct spatial solve (Sec. 2-3).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_timestep.py``:
  * on a generalised eigenvector K v = mu M v the scheme gives exactly
    u_n = (1 + kappa dt mu)^{-n} v;
  * the step matches a dense numpy.linalg.solve on a tiny case;
  * the manufactured solution u = sin(pi x) sin(pi y) cos t is approached at
    first order in dt.

The scheme (Sec. 2, Eq. (los) with theta = 1; Sec. 3):
    (M + kappa dt K) u^{k+1} = M u^k + dt f^{k+1},   k = 0 .. N_t-1,
which is the block forward solve of the space-time system A u = g of Sec. 3.
Reading: the source is evaluated at the new time level, f^{k+1} = c(t_{k+1}) fhat
(separable f = c(t) fhat(x) in every workload here).
"""
import numpy as np
from scipy.sparse.linalg import splu


class BackwardEuler:
    def __init__(self, M, K, kappa, dt):
        self.M = M.tocsr()
        self.K = K.tocsr()
        self.kappa = kappa
        self.dt = dt
        self.A = (self.M + kappa * dt * self.K).tocsc()
        self.lu = splu(self.A)

    def step(self, u, fvec=None):
        rhs = self.M @ u
        if fvec is not None:
            rhs = rhs + self.dt * fvec
        return self.lu.solve(rhs)


def sequential(M, K, kappa, T, Nt, u0, fhat=None, fcoef=None):
    """All time levels u_0..u_Nt of sequential backward Euler, shape (Nt+1, N).
    fcoef: callable t -> c(t), or an array of length Nt+1 (c at t_n)."""
    dt = T / Nt
    be = BackwardEuler(M, K, kappa, dt)
    U = np.zeros((Nt + 1, len(u0)))
    U[0] = u0
    for n in range(1, Nt + 1):
        fvec = None
        if fhat is not None:
            c = fcoef(n * dt) if callable(fcoef) else fcoef[n]
            fvec = c * fhat
        U[n] = be.step(U[n - 1], fvec)
    return U
