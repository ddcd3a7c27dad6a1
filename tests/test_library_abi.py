"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, and
exports every function include/fdlbm.h declares; the product path refuses to run without
CUDA (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdlbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for req in ("fdlbm_create", "fdlbm_step", "fdlbm_moments", "fdlbm_enthalpy_balance",
                "fdlbm_destroy", "fdlbm_last_error"):
        assert req in names


def test_library_exports_every_declared_symbol():
    from paper_1804_07588_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1804_07588_gb300 import fdlbm
    assert set(fdlbm.EXPORTS) <= set(declared_functions())


def test_last_error_without_gpu_is_safe():
    from paper_1804_07588_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.fdlbm_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.fdlbm_last_error(), bytes)


def test_solver_refuses_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1804_07588_gb300 import fdlbm, workloads
    with pytest.raises(RuntimeError):
        fdlbm.Solver(workloads.periodic_box(8, 8))
