"""p-multigrid spatial solver (Sec. 4, steps 1-5 and Fig. 5), plain FP64.

Test infrastructure (see ``oracle/__init__``).  Pinned by
``tests/test_oracle_pmg.py``:
  * ILUT with drop tolerance 0 and unlimited fill is the exact LU factorisation
    (L U reproduces A; one smoothing step then solves A x = b exactly);
  * ILUT(tau, fill) keeps at most ceil(fill*nnz) entries per row part and
    always keeps the diagonal; when the limit bites it keeps the largest
    |values|, exact ties going to the smaller column (a tiny matrix whose
    candidates are known by hand); on the 5-point Laplacian with fill = 1 it
    keeps exactly A's pattern;
  * the h-multigrid cycle is a W-cycle: its error propagation operator equals
    the one composed by hand from dense Gauss--Seidel, Galerkin and exact
    coarsest-solve operators with two coarse visits (three-level hierarchy);
  * lexicographic Gauss--Seidel equals the textbook element-by-element sweep
    (brute-force loop on a tiny grid);
  * the L2 transfers reproduce constants on the full basis:
    (M_p^L)^{-1} P 1 = 1 and (M_1^L)^{-1} P^T 1 = 1;
  * the bilinear prolongation is exact for bilinear functions (knot insertion);
  * the V-cycle converges to the sparse direct solution, and its contraction
    factor stays well below one for p = 2..5.

The method (Sec. 4):
  1. nu1 pre-smoothing steps  x <- x + S (b - A x),  S = (L U)^{-1} from ILUT;
  2. r_1 = I_p^1 (b - A x),  I_p^1 v = (M_1^L)^{-1} P^T v   (P = P_1^p of Eq. (PM));
  3. solve A_1 e_1 = r_1 approximately by ONE W-cycle of h-multigrid with
     Gauss--Seidel smoothing and a direct solve on the coarsest mesh (Fig. 5);
  4. x <- x + I_1^p e_1,  I_1^p v = (M_p^L)^{-1} P v;
  5. nu2 post-smoothing steps.

Readings of points the paper leaves open:
  * ILUT is Saad's dual-threshold ILUT in natural (lexicographic) order:
    entries below droptol * ||a_i||_2 are dropped, then the ceil(fill*nnz_L(a_i))
    largest strictly-lower and ceil(fill*nnz_U(a_i)) largest strictly-upper
    entries are kept (ties: larger |value| first, then smaller column); the
    diagonal is always kept.  Defaults droptol = 1e-12, fill = 1.
  * h-multigrid: prolongation = bilinear interpolation (knot insertion for
    p=1 splines), restriction = its transpose, coarse operators = Galerkin
    R A P; coarsen while the element count is even and above
    ``coarsest_nel`` (default 8, the coarsest mesh of Fig. 5); one forward
    lexicographic Gauss--Seidel sweep before and after the coarse correction;
    the coarse problem is visited twice (W-cycle, gamma = 2); the coarsest
    problem is solved by a dense Cholesky factorisation.
  * a spatial solve stops when ||b - A x||_2 <= tol ||b||_2 (checked before
    every cycle); b = 0 gives x = 0 without cycling.
"""
import heapq
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


# ---------------------------------------------------------------------------------
# ILUT
# ---------------------------------------------------------------------------------
def ilut(A, droptol=1e-12, fill=1.0):
    """Dual-threshold incomplete LU in natural order.

    Returns (L, U) as CSR: L strictly lower (unit diagonal implied), U upper
    with the diagonal.  Row i is eliminated with the already-final U rows of
    its pivots, pivots taken in increasing column order (fill-in pivots join
    as they appear).  The arithmetic is done one operation at a time in a
    fixed order:  w_k <- w_k / u_kk ; w_j <- w_j - w_k * u_kj.
    """
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    Lrows, Urows = [], []           # per row: (cols ndarray, vals ndarray)
    Udiag = np.zeros(n)
    for i in range(n):
        c0, c1 = A.indptr[i], A.indptr[i + 1]
        cols = A.indices[c0:c1]
        vals = A.data[c0:c1]
        # row 2-norm, summed in increasing column order
        s = 0.0
        for v in vals:
            s += float(v) * float(v)
        tau = droptol * math.sqrt(s)
        nl = int(np.sum(cols < i))
        nu = int(np.sum(cols > i))
        lfil_l = int(math.ceil(fill * nl))
        lfil_u = int(math.ceil(fill * nu))

        w = {int(c): float(v) for c, v in zip(cols, vals)}
        heap = [int(c) for c in cols if c < i]
        heapq.heapify(heap)
        seen = set(heap)
        while heap:
            k = heapq.heappop(heap)
            wk = w[k] / Udiag[k]
            if abs(wk) < tau:
                del w[k]
                continue
            w[k] = wk
            ucols, uvals = Urows[k]
            for j, ukj in zip(ucols, uvals):
                j = int(j)
                if j in w:
                    w[j] = w[j] - wk * float(ukj)
                else:
                    w[j] = 0.0 - wk * float(ukj)
                    if j < i and j not in seen:
                        heapq.heappush(heap, j)
                        seen.add(j)
        if i not in w:
            raise ZeroDivisionError(f"ILUT: structurally zero pivot in row {i}")
        diag = w[i]
        lower = [(j, v) for j, v in w.items() if j < i and abs(v) >= tau]
        upper = [(j, v) for j, v in w.items() if j > i and abs(v) >= tau]
        lower.sort(key=lambda t: (-abs(t[1]), t[0]))
        upper.sort(key=lambda t: (-abs(t[1]), t[0]))
        lower = sorted(lower[:lfil_l])
        upper = sorted(upper[:lfil_u])
        if diag == 0.0:
            raise ZeroDivisionError(f"ILUT: zero pivot in row {i}")
        Udiag[i] = diag
        Lrows.append((np.array([j for j, _ in lower], dtype=np.int64),
                      np.array([v for _, v in lower])))
        Urows.append((np.array([i] + [j for j, _ in upper], dtype=np.int64),
                      np.array([diag] + [v for _, v in upper])))
        # U row for later pivots: strictly-upper part only (diagonal used separately)
        Urows[-1] = (Urows[-1][0][1:], Urows[-1][1][1:])
    L = _rows_to_csr(Lrows, n)
    Uoff = _rows_to_csr(Urows, n)
    U = (Uoff + sp.diags(Udiag)).tocsr()
    U.sort_indices()
    return L, U


def _rows_to_csr(rows, n):
    indptr = np.zeros(n + 1, dtype=np.int64)
    for i, (c, _) in enumerate(rows):
        indptr[i + 1] = indptr[i] + len(c)
    indices = np.concatenate([c for c, _ in rows]) if n else np.zeros(0, np.int64)
    data = np.concatenate([v for _, v in rows]) if n else np.zeros(0)
    M = sp.csr_matrix((data, indices, indptr), shape=(n, n))
    M.sort_indices()
    return M


def level_schedule(L):
    """level(i) = 1 + max{ level(j) : j < i, L_ij != 0 } (0 when row i has no
    strictly-lower entries): the plain definition of a level schedule of a
    lower-triangular solve."""
    L = sp.csr_matrix(L)
    n = L.shape[0]
    lev = np.zeros(n, dtype=np.int64)
    for i in range(n):
        c = L.indices[L.indptr[i]:L.indptr[i + 1]]
        c = c[c < i]
        lev[i] = 0 if c.size == 0 else 1 + lev[c].max()
    return lev


# ---------------------------------------------------------------------------------
# h-multigrid at p = 1
# ---------------------------------------------------------------------------------
def prolongation_1d(nel_coarse):
    """Interior p=1 nodes of a mesh with nel_coarse elements -> interior nodes of
    the mesh with 2*nel_coarse elements.  A coarse hat is the sum
    1/2 phi_{2J-1} + phi_{2J} + 1/2 phi_{2J+1} of fine hats (knot insertion)."""
    nc = nel_coarse - 1
    nf = 2 * nel_coarse - 1
    P = np.zeros((nf, nc))
    for c in range(nc):
        J = c + 1                  # 1-based coarse node
        for node, wgt in ((2 * J - 1, 0.5), (2 * J, 1.0), (2 * J + 1, 0.5)):
            P[node - 1, c] = wgt
    return sp.csr_matrix(P)


def gauss_seidel(A, b, x):
    """One forward lexicographic Gauss--Seidel sweep:
    x_new = (D + L)^{-1} (b - U x_old), L/U the strict triangles of A."""
    A = sp.csr_matrix(A)
    lower = sp.tril(A, k=0, format="csr")
    upper = sp.triu(A, k=1, format="csr")
    return spsolve_triangular(lower, b - upper @ x, lower=True)


class HMG:
    """h-multigrid hierarchy on the p = 1 operator (Sec. 4, Fig. 5)."""

    def __init__(self, A1, nel, coarsest_nel=8):
        self.A = [sp.csr_matrix(A1)]
        self.P = []
        self.nel = [nel]
        while self.nel[-1] > coarsest_nel and self.nel[-1] % 2 == 0:
            P1 = prolongation_1d(self.nel[-1] // 2)
            P2 = sp.kron(P1, P1, format="csr")       # index ix + n*iy on both meshes
            Ac = (P2.T @ self.A[-1] @ P2).tocsr()
            self.P.append(P2)
            self.A.append(Ac)
            self.nel.append(self.nel[-1] // 2)
        self.chol = sla.cho_factor(self.A[-1].toarray(), lower=True)

    def cycle(self, k, b, x):
        """One W-cycle (gamma = 2) starting at level k."""
        if k == len(self.A) - 1:
            return sla.cho_solve(self.chol, b)
        A = self.A[k]
        x = gauss_seidel(A, b, x)
        r = b - A @ x
        rc = self.P[k].T @ r
        ec = np.zeros(rc.shape)
        ec = self.cycle(k + 1, rc, ec)
        ec = self.cycle(k + 1, rc, ec)
        x = x + self.P[k] @ ec
        x = gauss_seidel(A, b, x)
        return x


# ---------------------------------------------------------------------------------
# p-multigrid
# ---------------------------------------------------------------------------------
class PMG:
    """p-multigrid for A = M + c K at order p, coarse correction at p = 1."""

    def __init__(self, hi, lo, c, nu1=1, nu2=1, droptol=1e-12, fill=1.0, coarsest_nel=8):
        self.A = (hi.M + c * hi.K).tocsr()
        self.A.sort_indices()
        self.nu1, self.nu2 = nu1, nu2
        if hi.p > 1:
            self.A1 = (lo.M + c * lo.K).tocsr()
            self.P = hi.transfer_to(lo)
            self.MpL = hi.lumped
            self.M1L = lo.lumped
        else:
            self.A1 = self.A
            self.P = sp.identity(hi.N, format="csr")
            self.MpL = np.ones(hi.N)
            self.M1L = np.ones(hi.N)
        self.L, self.U = ilut(self.A, droptol, fill)
        self.hmg = HMG(self.A1, hi.nel, coarsest_nel)

    def smooth(self, b, x):
        r = b - self.A @ x
        y = spsolve_triangular(self.L, r, lower=True, unit_diagonal=True)
        z = spsolve_triangular(self.U, y, lower=False)
        return x + z

    def restrict(self, r):
        return (self.P.T @ r) / self.M1L

    def prolong(self, e1):
        return (self.P @ e1) / self.MpL

    def vcycle(self, b, x):
        for _ in range(self.nu1):
            x = self.smooth(b, x)
        r1 = self.restrict(b - self.A @ x)
        e1 = self.hmg.cycle(0, r1, np.zeros(r1.shape))
        x = x + self.prolong(e1)
        for _ in range(self.nu2):
            x = self.smooth(b, x)
        return x

    def solve(self, b, x0, tol=1e-10, max_cycles=50, ncycles=0):
        """Returns (x, cycles).  ncycles > 0: exactly that many V-cycles."""
        nb = np.linalg.norm(b)
        if nb == 0.0:
            return np.zeros_like(b), 0
        x = np.array(x0, dtype=np.float64, copy=True)
        if ncycles > 0:
            for _ in range(ncycles):
                x = self.vcycle(b, x)
            return x, ncycles
        cycles = 0
        while np.linalg.norm(b - self.A @ x) > tol * nb and cycles < max_cycles:
            x = self.vcycle(b, x)
            cycles += 1
        return x, cycles
