"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, and
exports every function include/fdlbm.h declares; the product path refuses to run without
CUDA (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    """Every function the headers under include/ declare."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdlbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


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


# C struct name in include/fdlbm.h -> ctypes mirror in the binding
_STRUCTS = {"fdlbm_geometry": "Geometry", "fdlbm_species": "Species", "fdlbm_transport": "Transport",
            "fdlbm_kinetics": "Kinetics", "fdlbm_fields": "Fields", "fdlbm_options": "Options",
            "fdlbm_info_t": "Info", "fdlbm_balance": "Balance"}


def test_binding_structs_match_header_layout(tmp_path):
    """Every ctypes mirror of an ABI struct has the size and field offsets the C compiler
    gives the struct in include/fdlbm.h (a plain C program compiled with gcc prints
    them), so argument marshalling cannot drift from the header."""
    import shutil
    import subprocess
    from paper_1804_07588_gb300 import fdlbm
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fdlbm.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        cls = getattr(fdlbm, pyname)
        lines.append(f'  printf("{pyname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{pyname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for ln in filter(None, out):
        pyname, what, value = ln.split()
        cls = getattr(fdlbm, pyname)
        got = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(value), f"{pyname}.{what}: ctypes {got}, C {value}"


def test_header_direction_order_is_the_oracles():
    """The velocity order include/fdlbm.h gives for fdlbm_populations is the one the FP64
    oracles use (the GPU population parity tests compare the two index by index)."""
    import re

    import numpy as np

    import oracle
    h = open(os.path.join(ROOT, "include", "fdlbm.h")).read()
    blk = h[h.index("Direction i moves along e_i"):h.index("fdlbm_status fdlbm_populations")]
    two, three = blk.split("D3Q19")
    d2 = np.array([[int(a), int(b)] for a, b in re.findall(r"\((-?\d),(-?\d)\)", two)])
    d3 = np.array([[int(a), int(b), int(c)] for a, b, c in re.findall(r"\((-?\d),(-?\d),(-?\d)\)", three)])
    assert d2.shape == (9, 2) and d3.shape == (19, 3)
    np.testing.assert_array_equal(d3, oracle.velocities3())
    # D2Q9: the odd part f(u) - f(-u) of the oracle's equilibrium for u along one axis has
    # the sign of e_i's component on that axis (zero where it is zero)
    for axis in range(2):
        u = [0.0, 0.0]
        u[axis] = 0.01
        odd = (oracle.equilibrium(1.0, u[0], u[1], 1.0, 1.0 / 3.0)
               - oracle.equilibrium(1.0, -u[0], -u[1], 1.0, 1.0 / 3.0))
        np.testing.assert_array_equal(np.sign(odd).astype(int), d2[:, axis])
