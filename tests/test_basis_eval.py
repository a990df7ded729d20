"""The library's host B-spline evaluation (iga_basis_eval, the code behind
iga_assemble's basis) against the oracle's Cox--de Boor recursion (Sec. 2): the
knot-span indices bit-exactly, and the values and derivatives bit-exactly too
(both sides evaluate the recursion in the same order, host code without FMA
contraction).  Runs on the CPU: the call needs no device."""
import numpy as np
import pytest

from oracle import bspline


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("nel", [1, 3, 16])
def test_spans_values_derivatives_match_oracle(B, p, nel):
    knots = bspline.open_uniform_knots(p, nel)
    x = np.concatenate([np.random.default_rng(p * 100 + nel).uniform(0.0, 1.0, 40),
                        np.unique(knots), [np.nextafter(1.0, 0.0), np.nextafter(0.5, 1.0)]])
    span, N, dN = B.basis_eval(p, nel, x)
    want_span = bspline._span_indicator(knots, x).argmax(axis=1)
    assert np.array_equal(span, want_span)
    full, dfull = bspline.basis(knots, p, x), bspline.basis_deriv(knots, p, x)
    rows = np.arange(x.size)[:, None]
    cols = span[:, None] - p + np.arange(p + 1)[None, :]
    assert np.array_equal(N, full[rows, cols])
    assert np.array_equal(dN, dfull[rows, cols])
    # and nothing outside the span's p+1 functions
    rest = full.copy()
    rest[rows, cols] = 0.0
    assert not rest.any()


def test_invalid_arguments(B):
    with pytest.raises(B.IgmError):
        B.basis_eval(2, 4, [1.5])
    with pytest.raises(B.IgmError):
        B.basis_eval(0, 4, [0.5])
    with pytest.raises(B.IgmError):
        B.basis_eval(3, 0, [0.5])
