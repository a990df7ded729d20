"""Host-side argument checks of the Python binding (no GPU needed): tensors
handed to the library must be CUDA tensors of the type the call reads."""
import pytest


def test_pointer_check_rejects_host_and_mistyped_tensors():
    torch = pytest.importorskip("torch")
    from paper_2107_05337_gb300 import binding as B
    with pytest.raises(TypeError):
        B._dptr_of(torch.zeros(4, dtype=torch.float32), torch.float32, "apply_f32")
    with pytest.raises(TypeError):
        B._dptr_of(torch.zeros(4, dtype=torch.float64), torch.float32, "apply_f32")


@pytest.mark.parametrize("method", ["solve", "solve_static"])
def test_solve_rejects_wrong_dtype_shape_or_device_before_any_launch(method):
    """pmg_vcycle and pmg_vcycle_static read and write nrhs * N doubles of B
    and X: a float32 pair, a pair with too few columns, mismatched shapes or
    host tensors are refused by the binding, before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_2107_05337_gb300 import binding as B
    g = B.PMG.__new__(B.PMG)     # no library handle: only the argument checks run
    g.N, g.h = 16, None
    f = getattr(g, method)
    bad = [
        (torch.zeros(2, 16, dtype=torch.float32), torch.zeros(2, 16, dtype=torch.float32)),
        (torch.zeros(2, 15, dtype=torch.float64), torch.zeros(2, 15, dtype=torch.float64)),
        (torch.zeros(2, 16, dtype=torch.float64), torch.zeros(3, 16, dtype=torch.float64)),
        (torch.zeros(16, dtype=torch.float64), torch.zeros(16, dtype=torch.float64)),
        (torch.zeros(2, 16, dtype=torch.float64), torch.zeros(2, 16, dtype=torch.float64)),
    ]
    for Bm, X in bad:
        with pytest.raises(TypeError):
            f(Bm, X)
