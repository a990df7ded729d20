"""Conjugate gradients with a diagonal (Jacobi) preconditioner: the spatial
solver the paper compares p-multigrid against (Sec. 5, CPU timings; Fig. 8
top; the p-dependence noted in Sec. 4 and 5), plain FP64.

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_cg.py``:
  * the k-th iterate minimises the A-norm of the error over the affine Krylov
    space x_0 + span{z_0, (D^-1 A) z_0, ..., (D^-1 A)^(k-1) z_0}, z_0 = D^-1 r_0
    (computed independently by a dense projection);
  * on a diagonal matrix the first iterate is exact;
  * the converged iterate equals a sparse direct solve;
  * at fixed mesh width the iteration count grows with p on the IgA matrices.

The iteration (preconditioned CG, z = D^-1 r with D = diag(A)):
  r = b - A x, z = D^-1 r, p = z;
  repeat: q = A p, alpha = (r, z) / (p, q), x += alpha p, r -= alpha q,
          stop if ||r||_2 <= tol ||b||_2, z = D^-1 r,
          beta = (r, z)_new / (r, z)_old, p = z + beta p.
"""
import numpy as np


def pcg_jacobi(A, b, x0=None, tol=1e-10, maxiter=10000, niter=0):
    """Returns (x, iterations).  niter > 0: exactly niter iterations."""
    A = A.tocsr()
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0
    r = b - A @ x
    if niter == 0 and np.linalg.norm(r) <= tol * nb:
        return x, 0
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while True:
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if niter > 0:
            if it >= niter:
                break
        elif np.linalg.norm(r) <= tol * nb or it >= maxiter:
            break
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def cg_factory(M, K, tol=1e-10, maxiter=10000, niter=0):
    """Spatial solver factory for oracle.mgrit.MGRIT: PCG on M + c K, warm start."""
    def make(level, c):
        A = (M + c * K).tocsr()
        return lambda rhs, guess: pcg_jacobi(A, rhs, guess, tol=tol, maxiter=maxiter, niter=niter)
    return make
