"""Univariate B-spline basis by the Cox--de Boor recursion (Sec. 2 of the paper).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_bspline.py``: the worked example of Fig. 1 (linear and
quadratic B-splines on {0,0,1,2,3,3} and {0,0,0,1,2,3,3,3}), partition of unity,
support and end interpolation (Sec. 2), derivatives against central differences.

Conventions
-----------
* A knot vector ``knots`` of length N+p+1 defines N functions phi_{i,p},
  i = 0..N-1 (0-based here; the paper counts from 1).
* phi_{i,0} is the indicator of the half-open span [xi_i, xi_{i+1}).  At the
  right end of the parameter domain every half-open span is empty, so the
  value there is taken from the last non-empty span (the usual closure; the
  paper's definition is silent on this point).
* In the recursion a term whose denominator (a zero-length knot span) vanishes
  is dropped (0/0 := 0).
"""
import numpy as np


def open_uniform_knots(p, nel, a=0.0, b=1.0):
    """Uniform knot vector on [a,b] with nel spans, end knots repeated p+1 times
    (Sec. 2: knot span size h = (b-a)/nel, C^{p-1} continuity, interpolatory ends)."""
    inner = [a + (b - a) * k / nel for k in range(1, nel)]
    return np.array([a] * (p + 1) + inner + [b] * (p + 1), dtype=np.float64)


def num_basis(knots, p):
    return len(knots) - p - 1


def _span_indicator(knots, x):
    """phi_{i,0}(x) for all i: shape (len(x), len(knots)-1)."""
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nspan = len(knots) - 1
    B = np.zeros((x.size, nspan))
    for i in range(nspan):
        B[:, i] = (knots[i] <= x) & (x < knots[i + 1])
    # right end point: use the last non-empty span
    last = max(i for i in range(nspan) if knots[i + 1] > knots[i])
    at_end = x >= knots[-1]
    B[at_end, :] = 0.0
    B[at_end, last] = 1.0
    return B


def basis(knots, p, x):
    """All phi_{i,p}(x).  Returns array (len(x), N) with N = len(knots)-p-1.

    Cox--de Boor (Sec. 2):
        phi_{i,q}(x) = (x - xi_i)/(xi_{i+q} - xi_i) phi_{i,q-1}(x)
                     + (xi_{i+q+1} - x)/(xi_{i+q+1} - xi_{i+1}) phi_{i+1,q-1}(x)
    """
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    B = _span_indicator(knots, x)
    for q in range(1, p + 1):
        nq = len(knots) - q - 1
        Bn = np.zeros((x.size, nq))
        for i in range(nq):
            d1 = knots[i + q] - knots[i]
            d2 = knots[i + q + 1] - knots[i + 1]
            term = np.zeros(x.size)
            if d1 > 0.0:
                term += (x - knots[i]) / d1 * B[:, i]
            if d2 > 0.0:
                term += (knots[i + q + 1] - x) / d2 * B[:, i + 1]
            Bn[:, i] = term
        B = Bn
    return B


def basis_deriv(knots, p, x):
    """First derivatives d/dx phi_{i,p}(x), shape (len(x), N).

    Differentiating the recursion gives the textbook identity
        phi'_{i,p} = p/(xi_{i+p}-xi_i) phi_{i,p-1} - p/(xi_{i+p+1}-xi_{i+1}) phi_{i+1,p-1}
    (again with 0/0 := 0).
    """
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = num_basis(knots, p)
    D = np.zeros((x.size, n))
    if p == 0:
        return D
    Bm = basis(knots, p - 1, x)  # N+1 functions of degree p-1
    for i in range(n):
        d1 = knots[i + p] - knots[i]
        d2 = knots[i + p + 1] - knots[i + 1]
        if d1 > 0.0:
            D[:, i] += p / d1 * Bm[:, i]
        if d2 > 0.0:
            D[:, i] -= p / d2 * Bm[:, i + 1]
    return D


def gauss_legendre(nq, a, b):
    """nq-point Gauss--Legendre rule mapped to [a,b] (numpy's leggauss)."""
    t, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (b - a) * t + 0.5 * (a + b), 0.5 * (b - a) * w


def elements(knots):
    """Non-empty knot spans [(lo, hi), ...] in increasing order."""
    u = np.unique(knots)
    return [(u[k], u[k + 1]) for k in range(len(u) - 1)]
