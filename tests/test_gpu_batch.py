"""GPU: an uneven batch of independent MGRIT problems (different orders,
meshes, time grids, kappa, geometries) run concurrently by
mgrit_run_batched gives, for every member, exactly the result of its own
mgrit_run, and the member results match the oracle."""
import numpy as np
import pytest

from oracle import assembly, geometry, timestep
from paper_2107_05337_gb300 import inputs

pytestmark = pytest.mark.gpu

MEMBERS = [  # p, nel, Nt, kappa, geometry, m
    (2, 16, 64, 0.3, "unit_square", 4),
    (3, 32, 128, 2.0, "unit_square", 4),
    (4, 16, 256, 1.0, "unit_square", 4),
    (5, 8, 32, 5.0, "unit_square", 4),
    (2, 32, 100, 0.1, "unit_square", 4),
    (3, 8, 64, 1.5, "quarter_annulus", 8),
]


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_05337_gb300 import binding
    binding.lib()
    return binding


def _u0fn(seed):
    k, l, a = inputs.fourier_modes(seed=seed)
    return lambda xi, eta, x, y: sum(a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta)
                                     for s in range(len(a)))


def test_batch_equals_individual_runs_and_oracle(B):
    import torch
    probs, handles, u0s = [], [], []
    for i, (p, nel, Nt, kappa, geom, m) in enumerate(MEMBERS):
        pr = B.Problem(p, nel, geom, kappa=kappa)
        probs.append(pr)
        u0s.append(pr.project(_u0fn(100 + i)))
        handles.append(B.MGRIT(pr, T=0.5, Nt=Nt, m=m, tol=1e-11,
                               pmg=dict(tol=1e-12, precision=1 if i % 2 else 0)))
    ref = []
    for h, u0 in zip(handles, u0s):
        U, st, _ = h.run(u0)
        ref.append((U.cpu().numpy(), st))
    Us, stats, lat, status = B.mgrit_run_batched(handles, u0s)
    assert status == 0
    for i, (U, st) in enumerate(zip(Us, stats)):
        np.testing.assert_array_equal(U.cpu().numpy(), ref[i][0])
        assert st["iters"] == ref[i][1]["iters"]
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    # two members against the oracle's sequential backward Euler
    for i in (0, 5):
        p, nel, Nt, kappa, geom, m = MEMBERS[i]
        d = assembly.Discretisation(p, nel, geometry.get(geom))
        seq = timestep.sequential(d.M, d.K, kappa, 0.5, Nt, d.project(_u0fn(100 + i)))
        U = Us[i].cpu().numpy()
        assert np.linalg.norm(U - seq) / np.linalg.norm(seq) < 1e-9, i


def test_batch_rejects_repeated_handle(B):
    pr = B.Problem(2, 8)
    h = B.MGRIT(pr, T=0.5, Nt=16)
    u0 = pr.project(_u0fn(1))
    with pytest.raises(B.IgmError):
        B.mgrit_run_batched([h, h], [u0, u0])


S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
C = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)

DEVICE_MEMBERS = [  # p, nel, Nt, kappa, geometry, m, extra MGRIT options, source
    (2, 16, 64, 0.3, "unit_square", 4, {}, True),
    (3, 32, 128, 2.0, "unit_square", 4, dict(coarse_cycles=1), False),
    (4, 16, 256, 1.0, "unit_square", 4, dict(cycle="F"), True),
    (5, 8, 30, 5.0, "unit_square", 4, dict(cycle="W"), False),       # partial intervals
    (2, 32, 100, 0.1, "unit_square", 4, dict(relax=0, max_iter=80), False),
    (3, 8, 64, 1.5, "quarter_annulus", 8, {}, False),
    (2, 8, 4, 1.0, "unit_square", 4, {}, False),                      # one time level
]


@pytest.mark.parametrize("precision", [1, 0])
def test_device_scheduled_batch_equals_individual_runs(B, precision):
    """mgrit_run_batched_device (one persistent launch, device-side stopping
    tests) gives every member exactly its own mgrit_run: iterate, iteration
    count and residual history bit for bit, across orders, meshes, time grids,
    kappa, both maps, V/F/W cycles, F- and FCF-relaxation, coarse-cycle
    limits, sources and a single-level member."""
    import torch
    handles, u0s, fhats, fcoefs = [], [], [], []
    for i, (p, nel, Nt, kappa, geom, m, extra, src) in enumerate(DEVICE_MEMBERS):
        pr = B.Problem(p, nel, geom, kappa=kappa)
        u0s.append(pr.project(_u0fn(200 + i)))
        fhats.append(pr.load_vector(S) if src else None)
        fcoefs.append(np.array([C(n * 0.5 / Nt) for n in range(Nt + 1)]) if src else None)
        handles.append(B.MGRIT(pr, T=0.5, Nt=Nt, m=m, tol=1e-11,
                               pmg=dict(tol=1e-12, precision=precision), **extra))
    ref = []
    for h, u0, fh, fc in zip(handles, u0s, fhats, fcoefs):
        U, st, _ = h.run(u0, fh, fc)
        ref.append((U.cpu().numpy(), st))
    Us, stats, lat, status = B.mgrit_run_batched(handles, u0s, fhats, fcoefs, device=True)
    assert status == 0
    for i, (U, st) in enumerate(zip(Us, stats)):
        np.testing.assert_array_equal(U.cpu().numpy(), ref[i][0], err_msg=str(i))
        assert st["iters"] == ref[i][1]["iters"], i
        np.testing.assert_array_equal(st["res_hist"], ref[i][1]["res_hist"], err_msg=str(i))
        assert st["launches"] == 1
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    # and a second batch on the same handles (warm state) again
    Us2, stats2, _, status = B.mgrit_run_batched(handles, u0s, fhats, fcoefs, device=True)
    assert status == 0
    for i in range(len(handles)):
        np.testing.assert_array_equal(Us2[i].cpu().numpy(), ref[i][0])


def test_device_batch_rejects_mixed_precision(B):
    pr = B.Problem(2, 8)
    h0 = B.MGRIT(pr, T=0.5, Nt=16, pmg=dict(precision=0))
    h1 = B.MGRIT(pr, T=0.5, Nt=16, pmg=dict(precision=1))
    u0 = pr.project(_u0fn(1))
    with pytest.raises(B.IgmError):
        B.mgrit_run_batched([h0, h1], [u0, u0], device=True)
