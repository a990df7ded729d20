"""Every sweep layout the setup can choose (pmg_opts.layout forces one; the
autotuner picks among the same six), at the full grid sizes of the benchmarked
workloads, against the oracle's p-multigrid cycle (Sec. 4, steps 1-5):

* FP64 form, fixed cycle counts: the GPU iterate equals the oracle's to 1e-10;
* mixed form, one fixed refinement step: equal to the oracle's FP64 cycle to
  the FP32 rounding of the correction (2e-5 relative);
* mixed form to tolerance: equal to the sparse direct solution to 1e-10.

Grids: unit square with 64 x 64 elements (n = 66 .. 69 unknowns per grid row,
p = 2..5, the heat_c2 sizes) and the quarter annulus with 128 x 128 elements
at p = 4 (n = 130, annulus_c3).  A layout that does not fit in shared memory
for a problem is refused by the setup (IGM_ERR_ARG) and skipped; every
problem must admit at least two layouts in each form."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from oracle import assembly, geometry, pmg
from paper_2107_05337_gb300 import inputs

pytestmark = pytest.mark.gpu

LAYOUTS = (1, 2, 3, 4, 5, 6)
CASES = [("unit_square", 2, 64, 1.0 / 256), ("unit_square", 3, 64, 1.0 / 256),
         ("unit_square", 4, 64, 16.0 / 256), ("unit_square", 5, 64, 1.0 / 256),
         ("quarter_annulus", 4, 128, 1.0 / 1024)]

_ORACLE = {}


@pytest.fixture(scope="module")
def B():
    from paper_2107_05337_gb300 import binding
    binding.lib()
    return binding


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _oracle(geom, p, nel, c):
    key = (geom, p, nel, c)
    if key not in _ORACLE:
        hi, lo = assembly.problem(p, nel, geometry.get(geom))
        _ORACLE[key] = pmg.PMG(hi, lo, c)
    return _ORACLE[key]


def _setup(B, prob, c, **opts):
    try:
        return B.PMG(prob, c, **opts)
    except B.IgmError as e:
        assert e.status == -1 and "does not fit" in str(e), e
        return None


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("geom,p,nel,c", CASES)
def test_every_layout_fixed_cycles_fp64(B, geom, p, nel, c):
    prob = B.Problem(p, nel, geom)
    P = _oracle(geom, p, nel, c)
    Bm = inputs.random_block(61, prob.N, 2)
    X0 = inputs.random_block(62, prob.N, 2, scale=0.1)
    want = [P.solve(Bm[k], X0[k], ncycles=2)[0] for k in range(2)]
    ran = []
    for layout in LAYOUTS:
        g = _setup(B, prob, c, precision=0, layout=layout)
        if g is None:
            continue
        team, _, arena, staged = g.layout()
        assert team == (128 if layout <= 3 else 256)
        assert (arena, staged) == ((1, 0), (0, 1), (0, 0))[(layout - 1) % 3]
        Xg = _cuda(X0)
        cyc, _ = g.solve(_cuda(Bm), Xg, ncycles=2)
        assert np.all(cyc == 2)
        Xg = Xg.cpu().numpy()
        for k in range(2):
            assert _rel(Xg[k], want[k]) < 1e-10, (layout, k)
        ran.append(layout)
    assert len(ran) >= 2, ran


@pytest.mark.parametrize("geom,p,nel,c", CASES)
def test_every_layout_mixed_form(B, geom, p, nel, c):
    prob = B.Problem(p, nel, geom)
    P = _oracle(geom, p, nel, c)
    Bm = inputs.random_block(63, prob.N, 2)
    one = [P.solve(Bm[k], np.zeros(prob.N), ncycles=1)[0] for k in range(2)]
    lu = splu(sp.csc_matrix(P.A))
    direct = [lu.solve(Bm[k]) for k in range(2)]
    ran = []
    for layout in LAYOUTS:
        g = _setup(B, prob, c, precision=1, tol=1e-12, layout=layout)
        if g is None:
            continue
        X = _cuda(np.zeros_like(Bm))
        g.solve(_cuda(Bm), X, ncycles=1)
        X = X.cpu().numpy()
        for k in range(2):
            assert _rel(X[k], one[k]) < 2e-5, (layout, k)
        X = _cuda(np.zeros_like(Bm))
        cyc, _ = g.solve(_cuda(Bm), X)
        X = X.cpu().numpy()
        for k in range(2):
            assert _rel(X[k], direct[k]) < 1e-10, (layout, k, cyc)
        ran.append(layout)
    assert len(ran) >= 2, ran


def test_autotuned_layout_is_one_of_the_forced_ones(B):
    """The layout the autotuner keeps on the annulus_c3 grid is one of the six
    forced layouts above (so the parity tests cover it)."""
    prob = B.Problem(4, 128, "quarter_annulus")
    g = B.PMG(prob, 1.0 / 1024, precision=1, autotune=1)
    team, _, arena, staged = g.layout()
    assert team in (128, 256) and (arena, staged) in ((1, 0), (0, 1), (0, 0))
