"""Two-level and multilevel MGRIT for theta-scheme time stepping (Sec. 3,
with the theta of Sec. 2 Eq. (los)), plain FP64.

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_mgrit.py``:
  * the converged MGRIT solution equals sequential time stepping (the block
    forward solve of A u = g, Sec. 3) to 1e-12;
  * one coarse interval (N_t = m) is exact after the first relaxation;
  * exactness propagation: with F-relaxation, after k iterations the C-points
    j <= k are exact (the parareal property); with FCF, C-points j <= 2k;
  * the two-level error contraction per iteration, measured in the M-norm on
    the C-points, stays below the eigenvalue bound of the two-level theory
    (Dobrev et al. 2017, cited by the paper):
    |lambda|^m |lambda^m - lambda_c| (1-|lambda_c|^{N_c}) / (1-|lambda_c|)
    with lambda = 1/(1+kappa dt mu), lambda_c = 1/(1+kappa m dt mu);
  * skipping the redundant first F-relaxation of a fine-level cycle (the
    F-points are already Phi-consistent after the interpolation) changes
    nothing when the spatial solves are exact.

The method (Sec. 3, the MGRIT algorithm box; ideal interpolation P):
  level l has time step dt_l = m^l dt and N_{l+1} = floor(N_l / m) steps: the
  C-points of level l are the multiples of m, and when m does not divide N_l
  the last N_l - m N_{l+1} points form a partial interval of F-points only
  (relaxed from the last C-point, never injected); on level l
  the step is  u_n = Phi_l(u_{n-1}) + g_n,  Phi_l = Psi_l R_l,
  Psi_l = (M + theta kappa dt_l K)^{-1}, R_l = M - (1-theta) kappa dt_l K
  (rediscretised on every level; theta = 1 is backward Euler, Sec. 3).  On the
  fine level the source enters the solve:
  Phi_0(u) + g_n = Psi_0 (R_0 u + dt (theta c(t_n) + (1-theta) c(t_{n-1})) fhat),
  u_0 = g_0 = the projected initial condition.

  cycle(l, kind):  if l is the coarsest level: solve A^(l) u = g^(l) by
             forward stepping; else
             FCF-relaxation on A^(l) u = g^(l);
             inject the C-point residual  r_j = g_{jm} + Phi_l(u_{jm-1}) - u_{jm}
             as the right-hand side g^(l+1)_j of the next level (u^(l+1) = 0);
             visit level l+1: once (V-cycle), as an F-cycle then a V-cycle
             (F-cycle), or twice with the same kind (W-cycle); the second
             visit starts from the first one's result;
             correct u_{jm} += u^(l+1)_j and F-relax (= ideal interpolation
             P = [-A_FF^{-1} A_FC; I_C]).

Readings of points the paper leaves open or prints garbled:
  * Correction scheme: the coarse right-hand side is the injected residual,
    i.e. the algorithm box's residual is g^(l) - A^(l) u^(l) (printed with
    g^(L)).  Coarse levels start from u^(l+1) = 0 on every visit.
  * The interpolation's inverse A_FF^{-1} (missing in the printed P) is an
    F-relaxation from the corrected C-points.
  * Level count: coarsen while the level has more than ``min_coarse`` steps,
    has at least one full interval (N_l >= m) and fewer than ``max_levels``
    levels exist.  A step count not divisible by m leaves a partial last
    interval of F-points (the coarsening XBraid, the paper's library, uses).
  * Stopping test: after the relaxation of iteration k, rho_k =
    sqrt(sum_j ||r_j||_2^2) over the fine-level C-points; stop when
    rho_k <= tol * rho_0 (the reported iteration count is k, the number of
    coarse corrections done).
  * Relaxation order: on the fine level, after the first iteration, the
    leading F-relaxation of FCF is skipped because the interpolation has just
    made the F-points Phi-consistent with the C-points (an exact no-op when
    the spatial solves are exact or run to a tolerance from a warm start).
  * Each spatial solve is warm-started from the current value at that time
    point of the part of u that the solve produces (u_n - g_n).
  * F- and W-cycles (named, not defined, in Sec. 5): the standard multigrid
    recursions above.  A repeated visit of the coarsest level (an exact
    forward solve of an unchanged system) is skipped.
"""
import numpy as np


def level_sizes(Nt, m, max_levels=30, min_coarse=4):
    sizes = [Nt]
    while len(sizes) < max_levels and sizes[-1] > min_coarse and sizes[-1] // m >= 1:
        sizes.append(sizes[-1] // m)
    return sizes


class MGRIT:
    """MGRIT for (M + theta kappa dt K) u^{n} = (M - (1-theta) kappa dt K) u^{n-1}
    + dt (theta c(t_n) + (1-theta) c(t_{n-1})) fhat.

    solver_factory(level, c) must return a callable
    solve(rhs, guess) -> (x, cycles) for the matrix M + c K.
    cycle: "V", "F" or "W" (the hierarchy of Sec. 5)."""

    def __init__(self, M, K, kappa, T, Nt, m, solver_factory, u0, fhat=None, fcoef=None,
                 max_levels=30, min_coarse=4, relax="FCF", skip_redundant_F=True, theta=1.0,
                 cycle="V"):
        assert cycle in ("V", "F", "W")
        self.M = M.tocsr()
        self.K = K.tocsr()
        self.theta = theta
        self.kind = cycle
        self.kappa = kappa
        self.Nt = Nt
        self.m = m
        self.sizes = level_sizes(Nt, m, max_levels, min_coarse)
        self.L = len(self.sizes) - 1
        self.dt = [T / Nt * m ** l for l in range(len(self.sizes))]
        self.solve = [solver_factory(l, theta * kappa * self.dt[l]) for l in range(len(self.sizes))]
        self.fhat = fhat
        self.fcoef = fcoef
        self.relax = relax
        self.skip = skip_redundant_F
        N = M.shape[0]
        self.W = [np.zeros((s + 1, N)) for s in self.sizes]
        self.g = [None] + [np.zeros((s + 1, N)) for s in self.sizes[1:]]
        self.W[0][0] = u0
        self.cycles = []          # V-cycles of every spatial solve, in order

    def _c(self, n):
        f = self.fcoef
        return f(n * self.dt[0]) if callable(f) else f[n]

    def u(self, l, n):
        return self.W[l][n] if l == 0 else self.W[l][n] + self.g[l][n]

    def phi(self, l, n):
        """Solve part of the step into point n of level l (warm start W_n)."""
        u = self.u(l, n - 1)
        rhs = self.M @ u
        if self.theta != 1.0:
            rhs = rhs - (1.0 - self.theta) * self.kappa * self.dt[l] * (self.K @ u)
        if l == 0 and self.fhat is not None:
            c = self.theta * self._c(n) + (1.0 - self.theta) * self._c(n - 1)
            rhs = rhs + self.dt[0] * c * self.fhat
        x, cyc = self.solve[l](rhs, self.W[l][n])
        self.cycles.append(cyc)
        return x

    def f_relax(self, l):
        m = self.m
        nint = self.sizes[l] // m
        for j in range(nint):
            for k in range(1, m):
                n = j * m + k
                self.W[l][n] = self.phi(l, n)
        for n in range(nint * m + 1, self.sizes[l] + 1):  # partial last interval
            self.W[l][n] = self.phi(l, n)

    def c_relax(self, l):
        m = self.m
        for j in range(self.sizes[l] // m):
            n = (j + 1) * m
            self.W[l][n] = self.phi(l, n)

    def residuals(self, l):
        m = self.m
        return [self.phi(l, (j + 1) * m) - self.W[l][(j + 1) * m]
                for j in range(self.sizes[l] // m)]

    def down(self, l, fresh):
        """Relaxation and residual on level l; writes g^(l+1); returns ||r||."""
        if fresh or not self.skip:
            self.f_relax(l)
        if self.relax == "FCF":
            self.c_relax(l)
            self.f_relax(l)
        R = self.residuals(l)
        g = self.g[l + 1]
        g[0] = 0.0
        for j, r in enumerate(R):
            g[j + 1] = r
        self.W[l + 1][:] = 0.0
        return np.sqrt(sum(float(np.dot(r, r)) for r in R))

    def up(self, l):
        m = self.m
        for j in range(1, self.sizes[l] // m + 1):
            self.W[l][j * m] += self.u(l + 1, j)
        self.f_relax(l)

    def cycle(self, l, kind=None):
        kind = kind or self.kind
        if l == self.L:
            for n in range(1, self.sizes[l] + 1):
                self.W[l][n] = self.phi(l, n)
            return
        self.down(l, fresh=True)
        self.visit(l + 1, kind)
        self.up(l)

    def visit(self, l, kind):
        """The coarse-level visits of one cycle of the given kind."""
        visits = {"V": ["V"], "F": ["F", "V"], "W": ["W", "W"]}[kind]
        if l == self.L:
            visits = visits[:1]
        for k in visits:
            self.cycle(l, k)

    def run(self, tol=1e-10, max_iter=50, callback=None):
        """Returns (U [Nt+1, N], iterations, residual history)."""
        if self.L == 0:
            for n in range(1, self.Nt + 1):
                self.W[0][n] = self.phi(0, n)
            return self.W[0], 0, []
        hist = []
        it = 0
        while True:
            rho = self.down(0, fresh=(it == 0))
            hist.append(rho)
            if callback is not None:
                callback(it, self)
            if rho == 0.0 or rho <= tol * hist[0] or it >= max_iter:
                break
            self.visit(1, self.kind)
            self.up(0)
            it += 1
        return self.W[0], it, hist


def direct_factory(M, K):
    from scipy.sparse.linalg import splu

    def make(level, c):
        lu = splu((M + c * K).tocsc())
        return lambda rhs, guess: (lu.solve(rhs), 0)
    return make


def pmg_factory(hi, lo, tol=1e-10, max_cycles=50, ncycles=0, coarse_cycles=0, **pmg_kw):
    """p-multigrid spatial solves; coarse_cycles > 0: exactly that many cycles
    per solve on the coarse time levels (an inexact coarse propagator)."""
    from .pmg import PMG

    def make(level, c):
        P = PMG(hi, lo, c, **pmg_kw)
        nc = coarse_cycles if (level > 0 and coarse_cycles > 0) else ncycles
        return lambda rhs, guess: P.solve(rhs, guess, tol=tol, max_cycles=max_cycles, ncycles=nc)
    return make
