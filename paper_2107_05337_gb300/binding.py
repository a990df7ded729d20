"""ctypes binding of ``libigamgrit.so`` (C ABI in include/igamgrit.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream.  If the
library is missing the calls raise -- there is no CPU fallback.
"""
import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_long, c_void_p

import numpy as np

from . import build as _build

_LIB = None


class IgmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"igamgrit status {status}: {msg}")
        self.status = status


class IgaDesc(ctypes.Structure):
    _fields_ = [("p", c_int), ("nel", c_int), ("nquad", c_int), ("geom", c_int),
                ("gdeg", c_int * 2), ("gn", c_int * 2), ("gctrl", POINTER(c_double)),
                ("kappa", c_double)]


class PmgOpts(ctypes.Structure):
    _fields_ = [("nu1", c_int), ("nu2", c_int), ("ilut_droptol", c_double),
                ("ilut_fill", c_double), ("hmg_coarsest_nel", c_int), ("precision", c_int),
                ("inner_cycles", c_int), ("tol", c_double), ("max_cycles", c_int),
                ("trace", c_int), ("solver", c_int), ("autotune", c_int), ("layout", c_int),
                ("hmg_fp64", c_int)]


class MgritOpts(ctypes.Structure):
    _fields_ = [("T", c_double), ("Nt", c_int), ("m", c_int), ("max_levels", c_int),
                ("min_coarse", c_int), ("relax", c_int), ("tol", c_double), ("max_iter", c_int),
                ("pmg", PmgOpts), ("initial_guess", c_int), ("graphs", c_int),
                ("profile", c_int), ("theta", c_double), ("cycle", c_int),
                ("priority", c_int), ("coarse_cycles", c_int), ("fused", c_int)]


class MgritStats(ctypes.Structure):
    _fields_ = [("iters", c_int), ("levels", c_int), ("res_hist", c_double * 256),
                ("vcyc_mean", c_double), ("solves", c_long), ("vcycles", c_long),
                ("seconds", c_double), ("setup_seconds", c_double), ("launches", c_long),
                ("coarse_fallback", c_int)]


EXPORTS = {
    "iga_assemble": (c_int, [POINTER(IgaDesc), POINTER(c_void_p)]),
    "iga_destroy": (None, [c_void_p]),
    "iga_sizes": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "iga_quadrature_points": (c_int, [c_void_p, POINTER(c_double)]),
    "iga_load_vector": (c_int, [c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "iga_project": (c_int, [c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "iga_apply_f32": (c_int, [c_void_p, c_int, c_double, c_int, c_void_p, c_void_p, c_long,
                              c_void_p]),
    "iga_basis_eval": (c_int, [c_int, c_int, c_int, POINTER(c_double), POINTER(c_int),
                               POINTER(c_double), POINTER(c_double)]),
    "iga_assemble_host": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_double)]),
    "iga_transfer_host": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                  POINTER(c_double)]),
    "iga_apply_f32_layout": (c_int, [c_int, c_int, c_long, POINTER(c_int)]),
    "iga_apply_f32_plan": (c_int, [c_int, c_int, c_int, c_int, c_int, c_long, POINTER(c_int)]),
    "pmg_block_tri_host": (c_int, [c_int, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_double),
                                   POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                   POINTER(c_double), POINTER(c_double)]),
    "pmg_hmg_host": (c_int, [c_void_p, c_double, c_int, c_int, POINTER(c_int), POINTER(c_int),
                             POINTER(c_double)]),
    "pmg_ilut_host": (c_int, [c_int, POINTER(c_int), POINTER(c_int), POINTER(c_double), c_double,
                              c_double, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                              POINTER(c_int), POINTER(c_double), POINTER(c_int), POINTER(c_int),
                              POINTER(c_double)]),
    "iga_apply": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_long, c_void_p]),
    "pmg_default_opts": (None, [POINTER(PmgOpts)]),
    "pmg_setup": (c_int, [c_void_p, c_double, POINTER(PmgOpts), POINTER(c_void_p)]),
    "pmg_destroy": (None, [c_void_p]),
    "pmg_vcycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, c_int, POINTER(c_int),
                           c_void_p]),
    "pmg_vcycle_static": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, c_int,
                                  POINTER(c_int), c_void_p]),
    "pmg_ilut_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, c_void_p]),
    "pmg_trace": (c_int, [c_void_p, POINTER(ctypes.c_longlong), c_int]),
    "pmg_ilut_factors": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                 POINTER(c_int), POINTER(c_double), POINTER(c_int),
                                 POINTER(c_int), POINTER(c_double)]),
    "mgrit_default_opts": (None, [POINTER(MgritOpts)]),
    "mgrit_create": (c_int, [c_void_p, POINTER(MgritOpts), POINTER(c_void_p)]),
    "mgrit_destroy": (None, [c_void_p]),
    "mgrit_run": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double), c_void_p,
                          POINTER(MgritStats), c_void_p]),
    "pmg_layout": (c_int, [c_void_p, POINTER(c_int)]),
    "mgrit_run_batched": (c_int, [c_int, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                  POINTER(c_void_p), POINTER(c_void_p), c_void_p,
                                  POINTER(ctypes.c_float), c_void_p]),
    "mgrit_run_batched_device": (c_int, [c_int, POINTER(c_void_p), POINTER(c_void_p),
                                         POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                         c_void_p, POINTER(ctypes.c_float), c_void_p]),
    "phic_create": (c_int, [c_int, c_int, ctypes.c_ulonglong, POINTER(c_void_p)]),
    "phic_destroy": (None, [c_void_p]),
    "phic_set_weights": (c_int, [c_void_p, POINTER(ctypes.c_float)]),
    "phic_get_weights": (c_int, [c_void_p, POINTER(ctypes.c_float), POINTER(c_int)]),
    "phic_apply": (c_int, [c_void_p, c_int, c_void_p, c_long, c_void_p, c_long, c_void_p]),
    "phic_train": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, c_int, c_int, c_double,
                           ctypes.c_ulonglong, POINTER(c_double), c_void_p]),
    "phic_grad": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_long, POINTER(c_double),
                          POINTER(ctypes.c_float), POINTER(ctypes.c_float), c_void_p]),
    "mgrit_set_coarse_propagator": (c_int, [c_void_p, c_void_p, c_double]),
    "mgrit_solve": (c_int, [c_void_p, POINTER(MgritOpts), c_void_p, c_void_p, POINTER(c_double),
                            c_void_p, POINTER(MgritStats), c_void_p]),
    "mgrit_profile": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                              POINTER(c_int), POINTER(ctypes.c_float), POINTER(c_long)]),
    "igm_wait_selftest": (c_int, [c_long, c_void_p]),
    "igm_grid_barrier_selftest": (c_int, [c_int, ctypes.c_longlong, c_int, c_void_p]),
    "igm_last_error": (ctypes.c_char_p, []),
    "igm_kernel_launches": (c_long, []),
}


def lib_path():
    return _build.LIB


def lib():
    """Load the library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2107_05337_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status):
    if status != 0:
        raise IgmError(status, lib().igm_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("igamgrit needs a CUDA device (no CPU fallback)")
    return torch


def _stream():
    return c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dptr(t):
    return c_void_p(t.data_ptr())


def _dptr_of(t, dtype, what):
    """Device pointer of a CUDA tensor of the given dtype; TypeError otherwise
    (the library reads the memory as that type)."""
    if not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{what}: expected a CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    return c_void_p(t.data_ptr())


def basis_eval(p, nel, x):
    """iga_basis_eval on host points x in [0, 1]: (span [nx] int32, N [nx, p+1],
    dN [nx, p+1]) of the order-p basis on the open uniform knots of nel
    elements; the nonzero functions at x[i] are span[i]-p .. span[i]."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    span = np.zeros(x.size, dtype=np.int32)
    N = np.zeros((x.size, p + 1))
    dN = np.zeros((x.size, p + 1))
    _check(lib().iga_basis_eval(p, nel, x.size, x.ctypes.data_as(POINTER(c_double)),
                                span.ctypes.data_as(POINTER(c_int)),
                                N.ctypes.data_as(POINTER(c_double)),
                                dN.ctypes.data_as(POINTER(c_double))))
    return span, N, dN


def ilut_host(A, droptol=1e-12, fill=1.0):
    """pmg_ilut_host on a scipy CSR matrix A: (L, U) as scipy CSR (L strictly
    lower, U upper with the diagonal), computed by the library's host code."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    n = A.shape[0]
    ptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    ip = lambda a: a.ctypes.data_as(POINTER(c_int))
    dp = lambda a: a.ctypes.data_as(POINTER(c_double))
    nl, nu = c_int(), c_int()
    _check(lib().pmg_ilut_host(n, ip(ptr), ip(col), dp(val), droptol, fill, ctypes.byref(nl),
                               ctypes.byref(nu), None, None, None, None, None, None))
    lp, lc, lv = np.zeros(n + 1, np.int32), np.zeros(max(nl.value, 1), np.int32), np.zeros(max(nl.value, 1))
    up, uc, uv = np.zeros(n + 1, np.int32), np.zeros(max(nu.value, 1), np.int32), np.zeros(max(nu.value, 1))
    _check(lib().pmg_ilut_host(n, ip(ptr), ip(col), dp(val), droptol, fill, None, None,
                               ip(lp), ip(lc), dp(lv), ip(up), ip(uc), dp(uv)))
    L = sp.csr_matrix((lv[:nl.value], lc[:nl.value], lp), shape=(n, n))
    U = sp.csr_matrix((uv[:nu.value], uc[:nu.value], up), shape=(n, n))
    return L, U


def block_tri_host(F, n, upper):
    """pmg_block_tri_host on a scipy CSR factor of an n x n grid: (off-block
    CSR, [n] list of dense n x n inverses of the grid rows' diagonal blocks)."""
    import scipy.sparse as sp
    F = sp.csr_matrix(F)
    N = n * n
    ptr = np.ascontiguousarray(F.indptr, dtype=np.int32)
    col = np.ascontiguousarray(F.indices, dtype=np.int32)
    val = np.ascontiguousarray(F.data, dtype=np.float64)
    ip = lambda a: a.ctypes.data_as(POINTER(c_int))
    dp = lambda a: a.ctypes.data_as(POINTER(c_double))
    nnz = c_int()
    _check(lib().pmg_block_tri_host(n, int(upper), ip(ptr), ip(col), dp(val), ctypes.byref(nnz),
                                    None, None, None, None))
    op = np.zeros(N + 1, np.int32)
    oc = np.zeros(max(nnz.value, 1), np.int32)
    ov = np.zeros(max(nnz.value, 1))
    inv = np.zeros(n * n * (n + 1) // 2)
    _check(lib().pmg_block_tri_host(n, int(upper), ip(ptr), ip(col), dp(val), None, ip(op),
                                    ip(oc), dp(ov), dp(inv)))
    off = sp.csr_matrix((ov[:nnz.value], oc[:nnz.value], op), shape=(N, N))
    blocks, per = [], n * (n + 1) // 2
    for b in range(n):
        pk, X = inv[b * per:(b + 1) * per], np.zeros((n, n))
        for r in range(n):
            if upper:
                base = r * n - r * (r - 1) // 2
                X[r, r:] = pk[base:base + n - r]
            else:
                X[r, :r + 1] = pk[r * (r + 1) // 2:r * (r + 1) // 2 + r + 1]
        blocks.append(X)
    return off, blocks


def quarter_annulus_net():
    """B-spline control net (degrees (3,1), 4 x 2 points) of the map
    F(xi, eta) = (1 + eta) C(xi), C the cubic Bezier quarter arc with control
    points (1,0), (1,k), (k,1), (0,1), k = 4(sqrt 2 - 1)/3."""
    k = 4.0 * (np.sqrt(2.0) - 1.0) / 3.0
    arc = np.array([[1.0, 0.0], [1.0, k], [k, 1.0], [0.0, 1.0]])
    ctrl = np.stack([arc * 1.0, arc * 2.0])  # [eta index][xi index][2]
    return (3, 1), (4, 2), np.ascontiguousarray(ctrl)


def _desc(p, nel, geom="unit_square", kappa=1.0, nquad=0):
    """iga_desc for the unit square or the quarter annulus; returns (desc, the
    control-net array the descriptor points into, or None)."""
    d = IgaDesc()
    d.p, d.nel, d.nquad, d.kappa = p, nel, nquad, kappa
    ctrl = None
    if geom == "unit_square":
        d.geom = 0
    elif geom == "quarter_annulus":
        deg, gn, net = quarter_annulus_net()
        d.geom = 1
        d.gdeg[0], d.gdeg[1] = deg
        d.gn[0], d.gn[1] = gn
        ctrl = np.ascontiguousarray(net.ravel())
        d.gctrl = ctrl.ctypes.data_as(POINTER(c_double))
    else:
        raise ValueError(geom)
    return d, ctrl


def assemble_host(p, nel, geom="unit_square", which="M", nquad=0):
    """iga_assemble_host: M or K as a scipy CSR matrix of the interior unknowns,
    or the lumped masses (which = 'lumped'), from the library's host assembly."""
    import scipy.sparse as sp
    d, ctrl = _desc(p, nel, geom, 1.0, nquad)
    w = {"M": 0, "K": 1, "lumped": 2}[which]
    n = c_int()
    _check(lib().iga_assemble_host(ctypes.byref(d), w, ctypes.byref(n), None))
    n = n.value
    N, q = n * n, 2 * p + 1
    out = np.zeros(N if w == 2 else N * q * q)
    _check(lib().iga_assemble_host(ctypes.byref(d), w, None, out.ctypes.data_as(POINTER(c_double))))
    if w == 2:
        return out
    i = np.arange(N)
    ix, iy = i % n, i // n
    rows, cols, vals = [], [], []
    for dy in range(-p, p + 1):
        for dx in range(-p, p + 1):
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < n) & (jy >= 0) & (jy < n)
            rows.append(i[ok])
            cols.append((jx + n * jy)[ok])
            vals.append(out[i[ok] * q * q + (dy + p) * q + (dx + p)])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def transfer_host(p, nel, geom="unit_square", nquad=0):
    """iga_transfer_host: the order-p x order-1 transfer matrix as scipy CSR."""
    import scipy.sparse as sp
    d, ctrl = _desc(p, nel, geom, 1.0, nquad)
    nnz = c_int()
    _check(lib().iga_transfer_host(ctypes.byref(d), ctypes.byref(nnz), None, None, None))
    n, n1 = nel + p - 2, nel - 1
    ptr = np.zeros(n * n + 1, dtype=np.int32)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1))
    _check(lib().iga_transfer_host(ctypes.byref(d), None, ptr.ctypes.data_as(POINTER(c_int)),
                                   col.ctypes.data_as(POINTER(c_int)),
                                   val.ctypes.data_as(POINTER(c_double))))
    return sp.csr_matrix((val[:nnz.value], col[:nnz.value], ptr), shape=(n * n, n1 * n1))


def hmg_host(p, nel, kappa_dt, geom="unit_square", coarsest_nel=8):
    """pmg_hmg_host: the order-1 operators of every h-level as scipy CSR."""
    import scipy.sparse as sp
    d, ctrl = _desc(p, nel, geom, 1.0, 0)
    nlev, n = c_int(), c_int()
    _check(lib().pmg_hmg_host(ctypes.byref(d), kappa_dt, coarsest_nel, 0, ctypes.byref(nlev),
                              None, None))
    out = []
    for lev in range(nlev.value):
        _check(lib().pmg_hmg_host(ctypes.byref(d), kappa_dt, coarsest_nel, lev, None,
                                  ctypes.byref(n), None))
        m = n.value
        st = np.zeros(m * m * 9)
        _check(lib().pmg_hmg_host(ctypes.byref(d), kappa_dt, coarsest_nel, lev, None, None,
                                  st.ctypes.data_as(POINTER(c_double))))
        i = np.arange(m * m)
        ix, iy = i % m, i // m
        rows, cols, vals = [], [], []
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                jx, jy = ix + dx, iy + dy
                ok = (jx >= 0) & (jx < m) & (jy >= 0) & (jy < m)
                rows.append(i[ok])
                cols.append((jx + m * jy)[ok])
                vals.append(st[i[ok] * 9 + (dy + 1) * 3 + (dx + 1)])
        out.append(sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                 shape=(m * m, m * m)))
    return out


def apply_f32_layout(n, p, smem_max=232448):
    """iga_apply_f32_layout as a dict (cap 0: the grid does not fit)."""
    out = (c_int * 7)()
    _check(lib().iga_apply_f32_layout(n, p, smem_max, out))
    return dict(zip(("cap", "ring", "J", "xs", "ns", "rows", "smem"), list(out)))


def apply_f32_plan(form, n, p, nrhs, sms=152, smem_max=232448):
    """iga_apply_f32_plan as a dict: form "strip" or "curved"."""
    k = {"strip": (1, ("SR", "threads", "smem", "strips", "groups")),
         "curved": (2, ("TR", "TC", "HR", "HC", "tiles", "groups"))}[form]
    out = (c_int * len(k[1]))()
    _check(lib().iga_apply_f32_plan(k[0], n, p, nrhs, sms, smem_max, out))
    return dict(zip(k[1], list(out)))


class Problem:
    """IgA discretisation (iga_assemble): order p, nel x nel elements."""

    def __init__(self, p, nel, geom="unit_square", kappa=1.0, nquad=0):
        L = lib()
        d, self._ctrl = _desc(p, nel, geom, kappa, nquad)
        h = c_void_p()
        _check(L.iga_assemble(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.p, self.nel, self.geom, self.kappa = p, nel, geom, kappa
        n, N, nqp = c_int(), c_int(), c_int()
        _check(L.iga_sizes(h, ctypes.byref(n), ctypes.byref(N), ctypes.byref(nqp)))
        self.n, self.N, self.nqp = n.value, N.value, nqp.value

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.iga_destroy(self.h)
            self.h = None

    def quadrature_points(self):
        pts = np.zeros((self.nqp, 4))
        _check(lib().iga_quadrature_points(self.h, pts.ctypes.data_as(POINTER(c_double))))
        return pts

    def _fq(self, fn):
        q = self.quadrature_points()
        return np.ascontiguousarray(fn(q[:, 0], q[:, 1], q[:, 2], q[:, 3]), dtype=np.float64)

    def load_vector(self, fn):
        """b_i = int f Phi_i for fn(xi, eta, x, y); returns a CUDA float64 tensor."""
        torch = _torch()
        fq = self._fq(fn)
        out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        _check(lib().iga_load_vector(self.h, fq.ctypes.data_as(POINTER(c_double)), _dptr(out),
                                     _stream()))
        return out

    def project(self, fn):
        """L2 projection of fn(xi, eta, x, y) onto the spline space."""
        torch = _torch()
        fq = self._fq(fn)
        out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        _check(lib().iga_project(self.h, fq.ctypes.data_as(POINTER(c_double)), _dptr(out),
                                 _stream()))
        return out

    def apply_f32(self, which, X, c=0.0):
        """Y = M X, K X or (M + c K) X (which = 'M', 'K', 'A') on FP32 columns X [nrhs, N]
        (sum factorisation on the unit square, assembled stencils on a curved map)."""
        torch = _torch()
        if X.dim() != 2:
            raise ValueError("apply_f32: X must be [nrhs, ld] with ld >= N")
        X = X.contiguous()
        px = _dptr_of(X, torch.float32, "apply_f32")
        Y = torch.empty_like(X)
        _check(lib().iga_apply_f32(self.h, {"M": 0, "K": 1, "A": 2}[which], c, X.shape[0],
                                   px, _dptr(Y), X.shape[1], _stream()))
        return Y

    def apply(self, which, X):
        """Y = M X (which='M') or K X (which='K') on columns X [nrhs, N] (CUDA float64)."""
        torch = _torch()
        X = X.contiguous()
        px = _dptr_of(X, torch.float64, "apply")
        Y = torch.empty_like(X)
        nrhs = X.shape[0] if X.dim() == 2 else 1
        _check(lib().iga_apply(self.h, 0 if which == "M" else 1, nrhs, px, _dptr(Y),
                               self.N, _stream()))
        return Y


def pmg_opts(**kw):
    o = PmgOpts()
    lib().pmg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class PMG:
    """p-multigrid hierarchy for A = M + kappa_dt K (pmg_setup)."""

    def __init__(self, problem, kappa_dt, **opts):
        self.problem = problem
        self.opts = pmg_opts(**opts)
        h = c_void_p()
        _check(lib().pmg_setup(problem.h, kappa_dt, ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h
        self.N = problem.N

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.pmg_destroy(self.h)
            self.h = None

    def _columns(self, B, X, what):
        """Device pointers of the column blocks B, X: contiguous CUDA float64
        tensors of the same shape [nrhs, N] (TypeError otherwise, before any
        launch: the kernels read and write nrhs * N doubles)."""
        import torch
        for t, nm in ((B, "B"), (X, "X")):
            if t.dtype != torch.float64:
                raise TypeError(f"{what}: {nm} must be float64, got {t.dtype}")
        if B.dim() != 2 or tuple(B.shape) != tuple(X.shape) or B.shape[1] != self.N:
            raise TypeError(f"{what}: B and X must both be [nrhs, {self.N}], got "
                            f"{tuple(B.shape)} and {tuple(X.shape)}")
        if not (B.is_contiguous() and X.is_contiguous()):
            raise TypeError(f"{what}: B and X must be contiguous")
        return _dptr_of(B, torch.float64, what + " B"), _dptr_of(X, torch.float64, what + " X")

    def solve(self, B, X, ncycles=0, check=True):
        """In-place solves on columns: B, X CUDA float64 [nrhs, N]; returns cycles per column."""
        pb, px = self._columns(B, X, "solve")
        nrhs = B.shape[0]
        cyc = (c_int * max(nrhs, 1))()
        st = lib().pmg_vcycle(self.h, nrhs, pb, px, self.N, ncycles, cyc, _stream())
        if check:
            _check(st)
        return np.array(cyc[:nrhs], dtype=np.int64), st

    def solve_static(self, B, X, ncycles=0, check=True):
        """As solve(), through pmg_vcycle_static (no device allocation)."""
        pb, px = self._columns(B, X, "solve_static")
        nrhs = B.shape[0]
        cyc = (c_int * max(nrhs, 1))()
        st = lib().pmg_vcycle_static(self.h, nrhs, pb, px, self.N, ncycles, cyc, _stream())
        if check:
            _check(st)
        return np.array(cyc[:nrhs], dtype=np.int64), st

    def layout(self):
        """(threads per sweep team, ring slots, arena in shared memory, staged vector)."""
        out = (c_int * 4)()
        _check(lib().pmg_layout(self.h, out))
        return tuple(out)

    def ilut_apply(self, R):
        torch = _torch()
        Z = torch.empty_like(R)
        _check(lib().pmg_ilut_apply(self.h, R.shape[0], _dptr(R), _dptr(Z), self.N, _stream()))
        return Z

    PHASES = ("residual64", "residual", "ilut", "restrict", "wcycle", "prolong", "rhs", "gs",
              "ilut_wait", "ilut_off", "ilut_diag", "gs_wait", "gs_row", "gs_scan")

    def trace(self, reset=True):
        """Accumulated SM clocks per solver phase (handle set up with trace=1)."""
        out = (ctypes.c_longlong * len(self.PHASES))()
        _check(lib().pmg_trace(self.h, out, 1 if reset else 0))
        return dict(zip(self.PHASES, list(out)))

    def factors(self):
        """(L, U) as scipy CSR matrices (host copies of the ILUT factors)."""
        import scipy.sparse as sp
        L = lib()
        nl, nu = c_int(), c_int()
        null_i, null_d = POINTER(c_int)(), POINTER(c_double)()
        _check(L.pmg_ilut_factors(self.h, ctypes.byref(nl), ctypes.byref(nu), null_i, null_i,
                                  null_d, null_i, null_i, null_d))
        N = self.N
        lp = np.zeros(N + 1, np.int32); lc = np.zeros(nl.value, np.int32); lv = np.zeros(nl.value)
        up_ = np.zeros(N + 1, np.int32); uc = np.zeros(nu.value, np.int32); uv = np.zeros(nu.value)
        P_i = lambda a: a.ctypes.data_as(POINTER(c_int))
        P_d = lambda a: a.ctypes.data_as(POINTER(c_double))
        _check(L.pmg_ilut_factors(self.h, None, None, P_i(lp), P_i(lc), P_d(lv), P_i(up_), P_i(uc),
                                  P_d(uv)))
        return (sp.csr_matrix((lv, lc, lp), shape=(N, N)),
                sp.csr_matrix((uv, uc, up_), shape=(N, N)))


CYCLES = {"V": 0, "F": 1, "W": 2}


def mgrit_opts(**kw):
    """mgrit_opts from keyword arguments; cycle may be given as "V", "F" or "W"."""
    o = MgritOpts()
    lib().mgrit_default_opts(ctypes.byref(o))
    pmg_kw = kw.pop("pmg", {})
    if isinstance(kw.get("cycle"), str):
        kw["cycle"] = CYCLES[kw["cycle"]]
    for k, v in kw.items():
        setattr(o, k, v)
    for k, v in pmg_kw.items():
        setattr(o.pmg, k, v)
    return o


def _stats(st):
    return dict(iters=st.iters, levels=st.levels,
                res_hist=list(st.res_hist[:st.iters + 1]), vcyc_mean=st.vcyc_mean,
                solves=st.solves, vcycles=st.vcycles, seconds=st.seconds,
                setup_seconds=st.setup_seconds, launches=st.launches,
                coarse_fallback=st.coarse_fallback)


class MGRIT:
    """MGRIT handle (mgrit_create / mgrit_run): setup once, solve many times."""

    def __init__(self, problem, **opts):
        self.problem = problem
        self.opts = mgrit_opts(**opts)
        h = c_void_p()
        _check(lib().mgrit_create(problem.h, ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h
        self.Nt = self.opts.Nt

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.mgrit_destroy(self.h)
            self.h = None

    def run(self, u0, fhat=None, fcoef=None, U=None, check=True):
        """u0, fhat: CUDA float64 [N]; fcoef: host [Nt+1].  Returns (U, stats, status)."""
        torch = _torch()
        if U is None:
            U = torch.empty((self.Nt + 1, self.problem.N), dtype=torch.float64, device="cuda")
        fc = None if fcoef is None else np.ascontiguousarray(fcoef, dtype=np.float64)
        st = MgritStats()
        status = lib().mgrit_run(self.h, _dptr(u0), _dptr(fhat) if fhat is not None else None,
                                 fc.ctypes.data_as(POINTER(c_double)) if fc is not None else None,
                                 _dptr(U), ctypes.byref(st), _stream())
        if check:
            _check(status)
        return U, _stats(st), status

    def set_coarse_propagator(self, phic, switch=0.5):
        """Two-level FAS with a learned coarse propagator (Phic), or None."""
        _check(lib().mgrit_set_coarse_propagator(self.h, phic.h if phic is not None else None,
                                                  switch))
        self._phic = phic

    def profile(self, cap=100000):
        """Per-launch records of the last run made with profile=1."""
        cnt = c_int()
        lv = (c_int * cap)(); gr = (c_int * cap)(); md = (c_int * cap)()
        ms = (ctypes.c_float * cap)(); cy = (c_long * cap)()
        _check(lib().mgrit_profile(self.h, cap, ctypes.byref(cnt), lv, gr, md, ms, cy))
        k = cnt.value
        return dict(level=np.array(lv[:k]), grid=np.array(gr[:k]), mode=np.array(md[:k]),
                    ms=np.array(ms[:k], dtype=np.float64), cycles=np.array(cy[:k]))


def _ld(T):
    """Row stride of a 2D tensor (a single row may carry stride 0 from NumPy)."""
    return T.stride(0) if T.shape[0] > 1 else T.shape[1]


class Phic:
    """Learned coarse propagator (phic_*): a four-layer 3 x 3 convolutional
    network with GELU on the n x n coefficient grid, BF16 kernels."""

    def __init__(self, n, channels=32, seed=0):
        h = c_void_p()
        _check(lib().phic_create(n, channels, seed, ctypes.byref(h)))
        self.h = h
        self.n, self.channels = n, channels

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.phic_destroy(self.h)
            self.h = None

    @property
    def weights(self):
        cnt = c_int()
        _check(lib().phic_get_weights(self.h, None, ctypes.byref(cnt)))
        w = np.zeros(cnt.value, dtype=np.float32)
        _check(lib().phic_get_weights(self.h, w.ctypes.data_as(POINTER(ctypes.c_float)),
                                      ctypes.byref(cnt)))
        return w

    @weights.setter
    def weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.weights.size
        _check(lib().phic_set_weights(self.h, w.ctypes.data_as(POINTER(ctypes.c_float))))

    def apply(self, U):
        """U: CUDA float64 [nb, n*n] -> Phi_c of every row."""
        torch = _torch()
        out = torch.empty_like(U)
        _check(lib().phic_apply(self.h, U.shape[0], _dptr(U), _ld(U), _dptr(out), _ld(out),
                                _stream()))
        return out

    def train(self, U0, U1, steps, batch=16, lr=1e-3, seed=0):
        """Pairs U0[b] -> U1[b] (CUDA float64 [np, n*n]); returns per-step losses."""
        loss = np.zeros(max(steps, 1))
        assert _ld(U0) == _ld(U1)
        _check(lib().phic_train(self.h, U0.shape[0], _dptr(U0), _dptr(U1), _ld(U0), steps,
                                batch, lr, seed, loss.ctypes.data_as(POINTER(c_double)),
                                _stream()))
        return loss[:steps]

    def grad(self, U0, U1, input_grad=True):
        """Loss and back-propagated gradients on the pairs U0[b] -> U1[b] (CUDA
        float64 [nb, n*n]) as one minibatch: (loss, weight gradient [count],
        gradient w.r.t. the normalised inputs [nb, n*n] or None)."""
        assert _ld(U0) == _ld(U1)
        nb = U0.shape[0]
        cnt = self.weights.size
        gw = np.zeros(cnt, dtype=np.float32)
        gx = np.zeros((nb, self.n * self.n), dtype=np.float32) if input_grad else None
        loss = c_double()
        _check(lib().phic_grad(self.h, nb, _dptr(U0), _dptr(U1), _ld(U0), ctypes.byref(loss),
                               gw.ctypes.data_as(POINTER(ctypes.c_float)),
                               gx.ctypes.data_as(POINTER(ctypes.c_float)) if input_grad else None,
                               _stream()))
        return loss.value, gw, gx


def mgrit_run_batched(handles, u0s, fhats=None, fcoefs=None, Us=None, check=True, device=False):
    """Concurrent MGRIT solves of independent problems: mgrit_run_batched
    (streams and a host scheduler), or with device=True
    mgrit_run_batched_device (one persistent launch).  handles: MGRIT
    objects; u0s, fhats: CUDA float64 [N_i] (fhats entries may be None);
    fcoefs: host arrays [Nt_i+1] or None.  Returns (Us, stats list, latencies
    in ms, status)."""
    torch = _torch()
    k = len(handles)
    if Us is None:
        Us = [torch.empty((h.Nt + 1, h.problem.N), dtype=torch.float64, device="cuda")
              for h in handles]
    arr = lambda xs: (c_void_p * k)(*[x if isinstance(x, int) or x is None else x for x in xs])
    hs = arr([h.h.value for h in handles])
    u0p = arr([u.data_ptr() for u in u0s])
    Up = arr([U.data_ptr() for U in Us])
    fh = None if fhats is None else arr([None if f is None else f.data_ptr() for f in fhats])
    keep = None
    fc = None
    if fcoefs is not None:
        keep = [None if f is None else np.ascontiguousarray(f, dtype=np.float64) for f in fcoefs]
        fc = arr([None if f is None else f.ctypes.data for f in keep])
    st = (MgritStats * k)()
    lat = (ctypes.c_float * k)()
    fn = lib().mgrit_run_batched_device if device else lib().mgrit_run_batched
    status = fn(k, hs, u0p, fh, fc, Up, st, lat, _stream())
    if check:
        _check(status)
    return Us, [_stats(x) for x in st], np.array(lat[:], dtype=np.float64), status


def mgrit_solve(problem, u0, fhat=None, fcoef=None, U=None, check=True, **opts):
    """One-shot MGRIT solve (mgrit_solve).  u0, fhat: CUDA float64 [N]; fcoef:
    host array [Nt+1] of c(t_n).  Returns (U [Nt+1, N] CUDA float64, stats, status)."""
    torch = _torch()
    o = mgrit_opts(**opts)
    if U is None:
        U = torch.empty((o.Nt + 1, problem.N), dtype=torch.float64, device="cuda")
    fc = None
    if fcoef is not None:
        fc = np.ascontiguousarray(fcoef, dtype=np.float64)
    st = MgritStats()
    status = lib().mgrit_solve(problem.h, ctypes.byref(o), _dptr(u0),
                               _dptr(fhat) if fhat is not None else None,
                               fc.ctypes.data_as(POINTER(c_double)) if fc is not None else None,
                               _dptr(U), ctypes.byref(st), _stream())
    if check:
        _check(status)
    return U, _stats(st), status


def wait_selftest(spins=1 << 16):
    """Status of igm_wait_selftest (IGM_ERR_TIMEOUT = -5 when the bound works)."""
    return lib().igm_wait_selftest(spins, _stream())


def grid_barrier_selftest(nctas=8, wait_cycles=1 << 22, hold=1):
    """Status of igm_grid_barrier_selftest (IGM_ERR_TIMEOUT = -5 with hold = 1
    when the bound works, 0 with hold = 0)."""
    return lib().igm_grid_barrier_selftest(nctas, wait_cycles, hold, _stream())


def kernel_launches():
    return lib().igm_kernel_launches()
