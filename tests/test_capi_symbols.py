"""The C-ABI library loads and exports every function include/igamgrit.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "igamgrit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:igm_status|void|const char\*|long)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2107_05337_gb300 import binding, build
    build.build()
    L = ctypes.CDLL(build.LIB)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    # the binding wraps exactly the declared entry points
    assert set(binding.EXPORTS) == set(declared)


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_2107_05337_gb300 import binding
    monkeypatch.setattr(binding, "_LIB", None)
    monkeypatch.setattr(binding, "lib_path", lambda: str(tmp_path / "missing.so"))
    try:
        binding.lib()
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("expected a RuntimeError")
