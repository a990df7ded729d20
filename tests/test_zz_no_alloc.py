"""pmg_vcycle_static: the spatial solve for callers that cannot allocate device
memory (their GPU memory is committed to their own pool, or an allocation
would synchronise the device inside a timed loop).  It must give the same
result as pmg_vcycle on the same inputs, call after call, while its scratch
lives in the library's static device buffer.  This file is collected last so
that a failure here does not hide the other tests' results."""
import numpy as np
import pytest

from paper_2107_05337_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _device_memory():
    """(free bytes of the device from cudaMemGetInfo, bytes reserved by the
    device's default stream-ordered memory pool, the one cudaMallocAsync
    draws on), read through the driver library."""
    import ctypes
    import torch
    free, _ = torch.cuda.mem_get_info()
    cu = ctypes.CDLL("libcuda.so.1")
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    reserved = ctypes.c_uint64()
    CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT = 5
    assert cu.cuMemPoolGetAttribute(pool, CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT,
                                    ctypes.byref(reserved)) == 0
    return free, reserved.value


@pytest.mark.parametrize("p,nel,precision", [(5, 64, 0), (3, 16, 1)])
def test_static_scratch_solve_matches_pmg_vcycle(p, nel, precision):
    import torch
    from paper_2107_05337_gb300 import binding as B
    prob = B.Problem(p, nel)
    g = B.PMG(prob, 1.0 / 256, precision=precision, tol=1e-12)
    Bm = torch.as_tensor(inputs.random_block(41, prob.N, 3), dtype=torch.float64, device="cuda")
    X0 = inputs.random_block(42, prob.N, 3, scale=0.1)
    for call in range(2):   # two calls in a row: the buffer keeps the previous contents
        Xa = torch.as_tensor(X0, dtype=torch.float64, device="cuda")
        Xb = Xa.clone()
        ca, _ = g.solve(Bm, Xa, ncycles=2)
        cb, _ = g.solve_static(Bm, Xb, ncycles=2)
        assert np.array_equal(ca, cb) and np.all(cb == 2), call
        assert _rel(Xb.cpu().numpy(), Xa.cpu().numpy()) < 1e-10, call
        # to-tolerance solves agree as well, with the same cycle counts
        Ya = torch.zeros_like(Bm)
        Yb = torch.zeros_like(Bm)
        ca, _ = g.solve(Bm, Ya)
        cb, _ = g.solve_static(Bm, Yb)
        assert np.array_equal(ca, cb), call
        assert _rel(Yb.cpu().numpy(), Ya.cpu().numpy()) < 1e-10, call


def test_static_scratch_rejects_oversize():
    import torch
    from paper_2107_05337_gb300 import binding as B
    prob = B.Problem(5, 64)
    g = B.PMG(prob, 1.0 / 256, precision=0)
    nrhs = 200   # 200 columns of FP64 working vectors exceed the 16 MiB buffer
    Bm = torch.zeros((nrhs, prob.N), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(Bm)
    _, st = g.solve_static(Bm, X, check=False)
    assert st == -1
    assert "static buffer holds" in B.lib().igm_last_error().decode()


def test_static_calls_allocate_no_device_memory():
    """After a first call (which may load the kernels' code), further calls
    leave the device's free memory and the default memory pool unchanged:
    nothing is allocated, neither by cudaMalloc nor by cudaMallocAsync."""
    import torch
    from paper_2107_05337_gb300 import binding as B
    prob = B.Problem(5, 64)   # FP64 working vectors too large for shared memory: the
    g = B.PMG(prob, 1.0 / 256, precision=0, tol=1e-12)   # static buffer holds them
    Bm = torch.as_tensor(inputs.random_block(43, prob.N, 4), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(Bm)
    g.solve_static(Bm, X, ncycles=1)
    torch.cuda.synchronize()
    before = _device_memory()
    for _ in range(3):
        X.zero_()
        g.solve_static(Bm, X)
    torch.cuda.synchronize()
    assert _device_memory() == before
