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
