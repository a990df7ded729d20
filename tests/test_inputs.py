"""The seeded synthetic inputs (paper_2107_05337_gb300/inputs.py, shared by the
oracle and the CUDA path): deterministic, and with the ranges and structure
their docstrings state."""
import numpy as np

from paper_2107_05337_gb300 import inputs


def test_fourier_modes_deterministic_distinct_and_scaled():
    k, l, a = inputs.fourier_modes()
    k2, l2, a2 = inputs.fourier_modes()
    assert np.array_equal(k, k2) and np.array_equal(l, l2) and np.array_equal(a, a2)
    assert len(set(zip(k, l))) == len(k) == 8
    assert k.min() >= 1 and l.min() >= 1 and k.max() <= 8 and l.max() <= 8
    # a_s (k_s^2 + l_s^2) are standard normals
    assert np.all(np.isfinite(a)) and np.abs(a * (k * k + l * l)).max() < 6.0
    assert not np.array_equal(a, inputs.fourier_modes(seed=1)[2])


def test_batch_members_ranges_and_determinism():
    ms = inputs.batch_members()
    assert ms == inputs.batch_members() and len(ms) == 64
    for m in ms:
        assert m["nel"] in (32, 64, 128) and 2 <= m["p"] <= 5
        assert m["Nt"] in (128, 256, 512, 1024, 2048) and m["m"] == 4 and m["T"] == 1.0
        assert 0.1 <= m["kappa"] <= 10.0
    # uneven: every mesh, order and step count occurs
    assert {m["nel"] for m in ms} == {32, 64, 128}
    assert {m["p"] for m in ms} == {2, 3, 4, 5}
    assert len({m["Nt"] for m in ms}) == 5


def test_workload_table():
    w = inputs.WORKLOADS
    assert w["heat_c2"]["p"] == [2, 3, 4, 5] and w["heat_c2"]["Nt"] == 256
    assert w["annulus_c3"]["geom"] == "quarter_annulus" and w["annulus_c3"]["m"] == 8
    assert w["learned_c4"]["max_levels"] == 2


def test_random_block_seeded():
    a = inputs.random_block(3, 10, 4, scale=2.0)
    assert a.shape == (4, 10)
    assert np.array_equal(a, 2.0 * np.random.default_rng(3).standard_normal((4, 10)))
