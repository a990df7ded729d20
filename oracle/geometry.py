"""Parametric geometry maps F: (0,1)^2 -> Omega (Sec. 2, geometry function F).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_assembly.py`` (mass-matrix sum equals the area of Omega,
computed independently by Green's theorem along the boundary).

* ``UnitSquare``: F = identity.
* ``QuarterAnnulus``: F(xi, eta) = (1 + eta) * C(xi), where C is the cubic
  Bezier arc through (1,0) and (0,1) with inner control points (1,k), (k,1),
  k = 4(sqrt(2)-1)/3 -- the standard cubic approximation of the unit quarter
  circle.  xi is the angular and eta the radial parameter, so Omega lies
  between radius ~1 and ~2.  The map is written here directly in Bernstein
  form (not as a B-spline control net) so that it is independent of the
  library's B-spline geometry evaluation.
"""
import numpy as np

BEZIER_K = 4.0 * (np.sqrt(2.0) - 1.0) / 3.0
ARC_CTRL = np.array([[1.0, 0.0], [1.0, BEZIER_K], [BEZIER_K, 1.0], [0.0, 1.0]])


class UnitSquare:
    name = "unit_square"
    affine = True

    def map(self, xi, eta):
        return np.asarray(xi, float), np.asarray(eta, float)

    def jacobian(self, xi, eta):
        """J[..., a, b] = d x_a / d xi_b."""
        xi = np.asarray(xi, float)
        J = np.zeros(xi.shape + (2, 2))
        J[..., 0, 0] = 1.0
        J[..., 1, 1] = 1.0
        return J

    def area(self):
        return 1.0


def _bernstein3(t):
    t = np.asarray(t, float)
    s = 1.0 - t
    return np.stack([s ** 3, 3 * s * s * t, 3 * s * t * t, t ** 3], axis=-1)


def _bernstein3_deriv(t):
    t = np.asarray(t, float)
    s = 1.0 - t
    return np.stack([-3 * s * s, 3 * s * s - 6 * s * t, 6 * s * t - 3 * t * t, 3 * t * t], axis=-1)


def arc(t):
    """C(t) and C'(t) for the cubic Bezier quarter arc; each shape t.shape + (2,)."""
    return _bernstein3(t) @ ARC_CTRL, _bernstein3_deriv(t) @ ARC_CTRL


class QuarterAnnulus:
    name = "quarter_annulus"
    affine = False

    def map(self, xi, eta):
        C, _ = arc(xi)
        r = 1.0 + np.asarray(eta, float)
        return r * C[..., 0], r * C[..., 1]

    def jacobian(self, xi, eta):
        C, dC = arc(xi)
        r = 1.0 + np.asarray(eta, float)
        J = np.zeros(np.shape(r) + (2, 2))
        J[..., 0, 0] = r * dC[..., 0]
        J[..., 1, 0] = r * dC[..., 1]
        J[..., 0, 1] = C[..., 0]
        J[..., 1, 1] = C[..., 1]
        return J

    def area_by_green(self, nq=20):
        """Area of Omega by Green's theorem, A = 1/2 * closed-line-integral (x dy - y dx),
        along the four boundary curves with Gauss quadrature (independent of the
        area-element integration used in assembly)."""
        t, w = np.polynomial.legendre.leggauss(nq)
        t = 0.5 * (t + 1.0)
        w = 0.5 * w
        C, dC = arc(t)
        outer = 4.0 * np.sum(w * (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0]))  # radius 2, counter-clockwise
        inner = 1.0 * np.sum(w * (C[:, 0] * dC[:, 1] - C[:, 1] * dC[:, 0]))  # radius 1, traversed back
        # the two straight radial edges lie on the coordinate axes: x dy - y dx = 0 there
        return 0.5 * (outer - inner)


def get(name):
    return {"unit_square": UnitSquare, "quarter_annulus": QuarterAnnulus}[name]()
