"""Pins of the oracle's Cox--de Boor basis (Sec. 2) against the paper's worked
example (Fig. 1) and the properties Sec. 2 states."""
import os

import numpy as np
import pytest

from oracle import bspline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_bsplines.txt")
KNOTS = {1: [0, 0, 1, 2, 3, 3], 2: [0, 0, 0, 1, 2, 3, 3, 3]}


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        deg, idx, iv, expr = [s.strip() for s in line.split("|")]
        lo, hi = (float(v) for v in iv.split())
        rows.append((int(deg), int(idx), lo, hi, expr))
    return rows


@pytest.mark.parametrize("deg", [1, 2])
def test_fig1_worked_example(deg):
    rows = [r for r in _golden() if r[0] == deg]
    B_all = None
    for _, idx, lo, hi, expr in rows:
        x = np.linspace(lo, hi, 41)[1:-1]          # open interval: no knot ambiguity
        B = bspline.basis(KNOTS[deg], deg, x)
        want = eval(expr, {"__builtins__": {}}, {"x": x}) * np.ones_like(x)
        np.testing.assert_allclose(B[:, idx], want, rtol=0, atol=1e-14)
    # every function of the figure is covered
    assert {r[1] for r in rows} == set(range(len(KNOTS[deg]) - deg - 1))


@pytest.mark.parametrize("p,nel", [(1, 3), (2, 5), (3, 7), (4, 6), (5, 9)])
def test_partition_of_unity_nonnegative_support(p, nel):
    knots = bspline.open_uniform_knots(p, nel)
    x = np.linspace(0.0, 1.0, 1001)
    B = bspline.basis(knots, p, x)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    assert B.min() >= -1e-15
    for i in range(B.shape[1]):
        inside = (x >= knots[i]) & (x < knots[i + p + 1])
        inside |= (x == 1.0) & (knots[i + p + 1] == 1.0)
        assert np.all(B[~inside, i] == 0.0)
    # interpolatory at both end points
    assert B[0, 0] == 1.0 and B[-1, -1] == 1.0
    assert np.count_nonzero(B[0]) == 1 and np.count_nonzero(B[-1]) == 1


@pytest.mark.parametrize("p", [2, 3, 4])
def test_derivatives_and_continuity(p):
    knots = bspline.open_uniform_knots(p, 5)
    x = np.linspace(0.013, 0.987, 77)
    h = 1e-6
    fd = (bspline.basis(knots, p, x + h) - bspline.basis(knots, p, x - h)) / (2 * h)
    np.testing.assert_allclose(bspline.basis_deriv(knots, p, x), fd, atol=2e-7 * p * p)
    # C^{p-1}: values and first derivatives continuous across interior knots
    for k in [0.2, 0.4, 0.6, 0.8]:
        eps = 1e-9
        for f in (bspline.basis, bspline.basis_deriv):
            left = f(knots, p, [k - eps])
            right = f(knots, p, [k + eps])
            np.testing.assert_allclose(left, right, atol=1e-6 * p * p * 10)


def test_span_count_and_knots():
    knots = bspline.open_uniform_knots(3, 4)
    assert list(knots) == [0, 0, 0, 0, 0.25, 0.5, 0.75, 1, 1, 1, 1]
    assert bspline.num_basis(knots, 3) == 7
    assert len(bspline.elements(knots)) == 4
