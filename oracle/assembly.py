"""Gauss-quadrature assembly of the IgA matrices and vectors (Sec. 2 and Sec. 4).

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_assembly.py``:
  * p=1 on the unit square reproduces the textbook Q1 stencils
    M = h^2/36 [1 4 1; 4 16 4; 1 4 1],  K = 1/3 [-1 -1 -1; -1 8 -1; -1 -1 -1];
  * the sum of all entries of the full-basis M equals the area of Omega
    (unit square: 1; quarter annulus: Green's theorem, ``geometry``);
  * full-basis K has zero row sums (constants are in the spline space);
  * M, K symmetric, M positive definite, interior K positive definite;
  * lumped mass of the full basis on the unit square equals the closed form
    prod_d (xi_{i+p+1} - xi_i)/(p+1);
  * the L2 projection converges at rate p+1 (``tests/test_oracle_convergence``).

Matrices (Sec. 2, Eq. (los) and the M, K definitions; Sec. 4 Eq. (PM)):
    M_ij = int_Omega Phi_i Phi_j,  K_ij = int_Omega grad Phi_i . grad Phi_j,
    P_ij = int_Omega Phi_{i,p} Phi_{j,1}   (transfer matrix, order p x order 1),
    M^L_ii = sum_j M_ij                   (row-sum lumping, Sec. 4).
The tensor-product basis is Phi_(a,b)(xi,eta) = phi_a(xi) phi_b(eta), numbered
a + nb*b (xi fastest).  Integrals are taken over the parameter domain with the
Jacobian of F: d Omega = |det J| d xi d eta, grad = J^{-T} grad_xi.

Readings of points the paper leaves open:
  * nq = p+1 Gauss points per direction per element for every matrix and
    vector of a problem of order p, including its p=1 matrices and P.
  * Dirichlet condition: the first and last univariate function in each
    direction are removed; N = (nel+p-2)^2 interior unknowns.
  * Lumped masses use the full row sum over all (boundary included) columns,
    then keep the interior rows.
  * P with Dirichlet: interior rows x interior columns of the full P.
"""
import numpy as np
import scipy.sparse as sp

from . import bspline


class Discretisation:
    """Full-basis matrices of one order p on one geometry, plus the interior
    (Dirichlet-eliminated) restrictions."""

    def __init__(self, p, nel, geom, nq=None):
        self.p = p
        self.nel = nel
        self.geom = geom
        self.nq = nq if nq is not None else p + 1
        self.knots = bspline.open_uniform_knots(p, nel)
        self.nb = bspline.num_basis(self.knots, p)          # functions per direction
        self.n = self.nb - 2                                 # interior per direction
        self.N = self.n * self.n
        self._quad_cache = None
        self.M_full, self.K_full = self._assemble_MK()
        self.interior = self._interior_index(self.nb)
        self.M = self.M_full[self.interior][:, self.interior].tocsr()
        self.K = self.K_full[self.interior][:, self.interior].tocsr()
        self.lumped_full = np.asarray(self.M_full.sum(axis=1)).ravel()
        self.lumped = self.lumped_full[self.interior]

    @staticmethod
    def _interior_index(nb):
        idx = [a + nb * b for b in range(1, nb - 1) for a in range(1, nb - 1)]
        return np.array(idx, dtype=np.int64)

    # -- quadrature on every element ------------------------------------------------
    def quadrature(self):
        """List over elements (ex, ey) of (xi_q, eta_q, weight_q*|detJ|, J, ...).

        For every element returns a dict with the tensor quadrature points
        (flattened, xi fastest), the physical points, the weights w_q |det J|,
        the inverse-transpose Jacobians and the element's first active basis
        index in each direction."""
        if self._quad_cache is not None:
            return self._quad_cache
        els = bspline.elements(self.knots)
        out = []
        for ey, (y0, y1) in enumerate(els):
            qy, wy = bspline.gauss_legendre(self.nq, y0, y1)
            for ex, (x0, x1) in enumerate(els):
                qx, wx = bspline.gauss_legendre(self.nq, x0, x1)
                XI, ETA = np.meshgrid(qx, qy)            # [iq_eta, iq_xi]
                XI = XI.ravel()
                ETA = ETA.ravel()
                W = np.outer(wy, wx).ravel()
                J = self.geom.jacobian(XI, ETA)
                detJ = np.linalg.det(J)
                JinvT = np.linalg.inv(J).transpose(0, 2, 1)
                X, Y = self.geom.map(XI, ETA)
                out.append(dict(ex=ex, ey=ey, xi=XI, eta=ETA, x=X, y=Y,
                                wdet=W * np.abs(detJ), JinvT=JinvT,
                                qx=qx, qy=qy))
        self._quad_cache = out
        return out

    def _tables_1d(self, knots, p):
        """Per element span e: (active function indices, values [nq, p+1],
        derivatives [nq, p+1]) of the univariate basis at that span's Gauss
        points; cached per (knots, p)."""
        key = (tuple(knots), p)
        cache = getattr(self, "_t1d", {})
        if key in cache:
            return cache[key]
        nb = bspline.num_basis(knots, p)
        tabs = []
        for (a0, a1) in bspline.elements(self.knots):
            qx, _ = bspline.gauss_legendre(self.nq, a0, a1)
            B = bspline.basis(knots, p, qx)
            D = bspline.basis_deriv(knots, p, qx)
            act = [a for a in range(nb) if np.any(B[:, a] != 0.0) or np.any(D[:, a] != 0.0)]
            tabs.append((np.array(act), B[:, act], D[:, act]))
        cache[key] = tabs
        self._t1d = cache
        return tabs

    def _local_basis(self, q, knots, p):
        """Values and parametric gradients of the functions active on element q;
        returns (global full-basis indices, values [nq2, nloc], grads [nq2, nloc, 2]).
        Point order: eta outer, xi inner (matches the meshgrid ravel in quadrature())."""
        nb = bspline.num_basis(knots, p)
        tabs = self._tables_1d(knots, p)
        ax, Bx, Dx = tabs[q["ex"]]
        ay, By, Dy = tabs[q["ey"]]
        # tensor products: local function (b, a) -> column b*len(ax) + a
        V = np.einsum("yb,xa->yxba", By, Bx).reshape(len(q["xi"]), -1)
        Gxi = np.einsum("yb,xa->yxba", By, Dx).reshape(len(q["xi"]), -1)
        Geta = np.einsum("yb,xa->yxba", Dy, Bx).reshape(len(q["xi"]), -1)
        idx = (ay[:, None] * nb + ax[None, :]).ravel()
        return idx, V, np.stack([Gxi, Geta], axis=-1)

    def _assemble_MK(self):
        rows, cols, mv, kv = [], [], [], []
        for q in self.quadrature():
            idx, V, G = self._local_basis(q, self.knots, self.p)
            # physical gradients: J^{-T} grad_xi
            Gp = np.einsum("qab,qib->qia", q["JinvT"], G)
            w = q["wdet"]
            Me = np.einsum("q,qi,qj->ij", w, V, V)
            Ke = np.einsum("q,qia,qja->ij", w, Gp, Gp)
            r, c = np.meshgrid(idx, idx, indexing="ij")
            rows.append(r.ravel()); cols.append(c.ravel())
            mv.append(Me.ravel()); kv.append(Ke.ravel())
        n2 = self.nb * self.nb
        rows = np.concatenate(rows); cols = np.concatenate(cols)
        M = sp.coo_matrix((np.concatenate(mv), (rows, cols)), shape=(n2, n2)).tocsr()
        K = sp.coo_matrix((np.concatenate(kv), (rows, cols)), shape=(n2, n2)).tocsr()
        M.sum_duplicates(); K.sum_duplicates()
        return M, K

    # -- vectors ----------------------------------------------------------------------
    def load_vector(self, fn):
        """b_i = int_Omega fn * Phi_i for interior i.  fn(xi, eta, x, y) -> values."""
        b = np.zeros(self.nb * self.nb)
        for q in self.quadrature():
            idx, V, _ = self._local_basis(q, self.knots, self.p)
            fq = fn(q["xi"], q["eta"], q["x"], q["y"])
            np.add.at(b, idx, V.T @ (q["wdet"] * fq))
        return b[self.interior]

    def project(self, fn):
        """Consistent L2 projection onto the interior spline space: M u = b (Sec. 3: the
        initial condition is projected onto the spline space)."""
        from scipy.sparse.linalg import spsolve
        return spsolve(self.M.tocsc(), self.load_vector(fn))

    def transfer_to(self, low, full=False):
        """P_ij = int Phi_{i,p} Phi_{j,low.p} over interior i (this order) and
        interior j (the order of ``low``, same knots spans and quadrature);
        ``full=True`` returns the matrix over the full bases."""
        assert low.nel == self.nel
        rows, cols, vals = [], [], []
        for q in self.quadrature():
            ih, Vh, _ = self._local_basis(q, self.knots, self.p)
            il, Vl, _ = self._local_basis(q, low.knots, low.p)
            Pe = np.einsum("q,qi,qj->ij", q["wdet"], Vh, Vl)
            r, c = np.meshgrid(ih, il, indexing="ij")
            rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Pe.ravel())
        P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.nb * self.nb, low.nb * low.nb)).tocsr()
        P.sum_duplicates()
        if full:
            return P
        return P[self.interior][:, low.interior].tocsr()

    def l2_error(self, u_interior, exact, nq_err=None):
        """|| u_h - exact ||_{L2(Omega)} with u_h the interior coefficient vector
        (boundary coefficients zero); exact(xi, eta, x, y).  Uses its own
        nq_err-point Gauss rule (default p+3) so that the error is not sampled
        only at the assembly rule's (superconvergent) points."""
        nq_err = nq_err or self.p + 3
        full = np.zeros(self.nb * self.nb)
        full[self.interior] = u_interior
        els = bspline.elements(self.knots)
        err2 = 0.0
        for ey, (y0, y1) in enumerate(els):
            qy, wy = bspline.gauss_legendre(nq_err, y0, y1)
            By = bspline.basis(self.knots, self.p, qy)
            for ex, (x0, x1) in enumerate(els):
                qx, wx = bspline.gauss_legendre(nq_err, x0, x1)
                Bx = bspline.basis(self.knots, self.p, qx)
                XI, ETA = np.meshgrid(qx, qy)
                XI = XI.ravel(); ETA = ETA.ravel()
                W = np.outer(wy, wx).ravel() * np.abs(np.linalg.det(self.geom.jacobian(XI, ETA)))
                C = full.reshape(self.nb, self.nb)          # [b (eta), a (xi)]
                uh = np.einsum("yb,ba,xa->yx", By, C, Bx).ravel()
                X, Y = self.geom.map(XI, ETA)
                e = uh - exact(XI, ETA, X, Y)
                err2 += np.sum(W * e * e)
        return np.sqrt(err2)


def problem(p, nel, geom, nq=None):
    """Order-p discretisation plus the order-1 one on the same knots and rule
    (used by p-multigrid; Sec. 4: the level p=1 is a rediscretisation)."""
    hi = Discretisation(p, nel, geom, nq=nq)
    lo = Discretisation(1, nel, geom, nq=hi.nq) if p > 1 else hi
    return hi, lo
