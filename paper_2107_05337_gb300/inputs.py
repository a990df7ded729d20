"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds only random draws and workload shape tables -- none of the
method's arithmetic (no basis, quadrature, assembly or solver code).  Random
numbers come from NumPy's PCG64 (``numpy.random.default_rng``).

Workloads (shapes of the paper's experiments, Sec. 5; sizes as stated here):
  * ``heat_c1``: unit square, p=2, 16 elements per direction, T=1, N_t=100,
    two-level MGRIT with m=4.
  * ``heat_c2``: unit square, h=1/64, p in {2,3,4,5}, T=1, N_t=256, multilevel
    MGRIT with m=4 down to at most 4 coarse steps.
  * ``annulus_c3``: quarter annulus (radii 1 and 2), p=4, 128 elements per
    direction, T=1, N_t=1024, f=0, multilevel MGRIT with m=8; initial condition
    a sum of 8 Fourier modes, see ``fourier_modes``.
The manufactured solution on the unit square is u = sin(pi x) sin(pi y) cos t
with kappa = 1, so f = (2 kappa pi^2 cos t - sin t) sin(pi x) sin(pi y).
"""
import numpy as np

SEED_ANNULUS = 20210712
SEED_BATCH = 20210714
SEED_LEARNED = 20210713


def fourier_modes(seed=SEED_ANNULUS, count=8, kmax=8):
    """``count`` distinct integer pairs (k, l) drawn uniformly from [1, kmax]^2 and
    amplitudes a_s ~ N(0,1) / (k_s^2 + l_s^2).  Returns (k, l, a) arrays."""
    rng = np.random.default_rng(seed)
    pairs = []
    while len(pairs) < count:
        k, l = (int(v) for v in rng.integers(1, kmax + 1, size=2))
        if (k, l) not in pairs:
            pairs.append((k, l))
    k = np.array([q[0] for q in pairs], dtype=np.float64)
    l = np.array([q[1] for q in pairs], dtype=np.float64)
    a = rng.standard_normal(count) / (k * k + l * l)
    return k, l, a


def random_block(seed, n, ncols, scale=1.0):
    """A dense [ncols, n] float64 block of standard normals (test right-hand sides)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((ncols, n))


WORKLOADS = {
    "heat_c1": dict(geom="unit_square", p=[2], nel=16, T=1.0, Nt=100, m=4, max_levels=2,
                    min_coarse=4, kappa=1.0, source="manufactured"),
    "heat_c2": dict(geom="unit_square", p=[2, 3, 4, 5], nel=64, T=1.0, Nt=256, m=4,
                    max_levels=30, min_coarse=4, kappa=1.0, source="manufactured"),
    "annulus_c3": dict(geom="quarter_annulus", p=[4], nel=128, T=1.0, Nt=1024, m=8,
                       max_levels=30, min_coarse=4, kappa=1.0, source="none"),
    "batch_c5": dict(members="batch_members()", source="none"),
    "learned_c4": dict(geom="unit_square", p=[3], nel=64, T=4.0, Nt=4096, m=8, max_levels=2,
                       kappa=1.0, source="none", train_ics=5, modes=16, seed=SEED_LEARNED),
}


def batch_members(seed=SEED_BATCH, count=64):
    """The uneven multi-problem batch: ``count`` independent heat problems on the
    unit square with h drawn from {1/32, 1/64, 1/128}, p from {2, 3, 4, 5}, N_t
    from {128, 256, 512, 1024, 2048}, kappa log-uniform on [0.1, 10], T = 1,
    f = 0, m = 4, and an initial condition of 16 random Fourier modes
    (``fourier_modes`` with a per-member seed).  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nel = int(rng.choice([32, 64, 128]))
        p = int(rng.integers(2, 6))
        Nt = int(rng.choice([128, 256, 512, 1024, 2048]))
        kappa = float(10.0 ** rng.uniform(-1.0, 1.0))
        modes_seed = int(rng.integers(0, 2 ** 31 - 1))
        out.append(dict(p=p, nel=nel, Nt=Nt, kappa=kappa, T=1.0, m=4, modes_seed=modes_seed))
    return out
