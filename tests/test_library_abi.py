"""CPU-side checks of the C-ABI library: it loads and exports every symbol include/mstopo.h
declares (no compute calls: those need a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mstopo.h")).read()
    return sorted(set(re.findall(r"\b(mstopo_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_symbols():
    from paper_1411_3923_gb300 import SYMBOLS
    assert sorted(SYMBOLS) == declared_symbols()


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1411_3923_gb300 import _build
    try:
        _build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    path = _build.build()
    import ctypes
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_invalid_problem_is_rejected_without_gpu_work():
    """mstopo_create validates its arguments before touching the device."""
    import ctypes
    import numpy as np
    import paper_1411_3923_gb300 as m
    from paper_1411_3923_gb300 import mstopo
    lib = m.load()
    fixed = np.zeros(2 * 9 * 5, np.uint8)
    d = mstopo._Problem(8, 4, 0.3, 1.0, 1e-9, 3.0, fixed.ctypes.data, 3, 4, 0.0, 1, 1e-8, 100, 0.0, None)
    h = ctypes.c_void_p()
    assert lib.mstopo_create(ctypes.byref(d), ctypes.byref(h)) == 1      # 8 % 3 != 0
    assert h.value is None
    assert b"invalid" in lib.mstopo_last_error(None)


@pytest.mark.parametrize("c_name,py_name", [("mstopo_problem", "_Problem"),
                                             ("mstopo_build_info", "_BuildInfo"),
                                             ("mstopo_solve_info", "_SolveInfo"),
                                             ("mstopo_stats", "_Stats"),
                                             ("mstopo_pde_desc", "_PdeDesc"),
                                             ("mstopo_opt_stage", "_OptStage"),
                                             ("mstopo_opt_record", "_OptRecord")])
def test_ctypes_structs_match_the_header_layout(tmp_path, c_name, py_name):
    """Every public struct of include/mstopo.h has the same size and field offsets in the
    binding's ctypes mirror: a C program compiled against the header prints them."""
    import ctypes
    import shutil
    import subprocess
    from paper_1411_3923_gb300 import mstopo
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    py = getattr(mstopo, py_name)
    fields = [f[0] for f in py._fields_]
    lines = [f'printf("size %zu\\n", sizeof({c_name}));']
    lines += [f'printf("{f} %zu\\n", offsetof({c_name}, {f}));' for f in fields]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"mstopo.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(py), (c_name, out["size"], ctypes.sizeof(py))
    for f in fields:
        assert int(out[f]) == getattr(py, f).offset, (c_name, f)


def test_unknown_preconditioner_kind_is_rejected():
    import ctypes
    import numpy as np
    import paper_1411_3923_gb300 as m
    from paper_1411_3923_gb300 import mstopo
    lib = m.load()
    fixed = np.zeros(2 * 9 * 9, np.uint8)
    # valid in every other field (8x8 elements, H 4: two coarse cells each way)
    for kind in (7, -1):
        d = mstopo._Problem(8, 8, 0.3, 1.0, 1e-9, 3.0, fixed.ctypes.data, 4, 4, 0.0, 1, 1e-8, 100,
                            0.0, None, 0, 0, 0.0, kind)
        h = ctypes.c_void_p()
        assert lib.mstopo_create(ctypes.byref(d), ctypes.byref(h)) == 1
        assert h.value is None


@pytest.mark.parametrize("patch_kernel,exec_flags", [(3, 0), (-1, 0), (0, 8), (0, -1)])
def test_unknown_patch_kernel_or_exec_flag_is_rejected(patch_kernel, exec_flags):
    """The kernel-path switches are problem fields and are validated before any GPU work."""
    import ctypes
    import numpy as np
    import paper_1411_3923_gb300 as m
    from paper_1411_3923_gb300 import mstopo
    lib = m.load()
    fixed = np.zeros(2 * 9 * 9, np.uint8)
    d = mstopo._Problem(8, 8, 0.3, 1.0, 1e-9, 3.0, fixed.ctypes.data, 4, 4, 0.0, 1, 1e-8, 100,
                        0.0, None, 0, 0, 0.0, 0, patch_kernel, exec_flags)
    h = ctypes.c_void_p()
    assert lib.mstopo_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert h.value is None


@pytest.mark.parametrize("krylov,restart", [(2, 0), (-1, 0), (1, -1), (1, 201)])
def test_unknown_krylov_method_or_restart_is_rejected(krylov, restart):
    """The outer method and the GMRES restart length are validated before any GPU work."""
    import ctypes
    import numpy as np
    import paper_1411_3923_gb300 as m
    from paper_1411_3923_gb300 import mstopo
    lib = m.load()
    fixed = np.zeros(2 * 9 * 9, np.uint8)
    d = mstopo._Problem(8, 8, 0.3, 1.0, 1e-9, 3.0, fixed.ctypes.data, 4, 4, 0.0, 1, 1e-8, 100,
                        0.0, None, 0, 0, 0.0, 0, 0, 0, krylov, restart)
    h = ctypes.c_void_p()
    assert lib.mstopo_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert h.value is None


@pytest.mark.parametrize("domain,nx,ny,rmin", [(3, 8, [8], 2.0), (1, 8, [8, 8], 2.0), (0, 0, [8], 2.0),
                                              (2, 8, [8, 0], 2.0), (0, 8, [8], 0.0)])
def test_invalid_pde_filter_is_rejected_without_gpu_work(domain, nx, ny, rmin):
    """mstopo_pde_filter_create validates the description before any device call."""
    import ctypes
    import numpy as np
    import paper_1411_3923_gb300 as m
    from paper_1411_3923_gb300 import mstopo
    lib = m.load()
    h = np.ascontiguousarray(ny, dtype=np.int32)
    d = mstopo._PdeDesc(domain, nx, len(ny), h.ctypes.data, rmin, 0.0, 0, None)
    f = ctypes.c_void_p()
    assert lib.mstopo_pde_filter_create(ctypes.byref(d), ctypes.byref(f)) == 1
    assert f.value is None
    assert b"invalid" in lib.mstopo_pde_filter_last_error(None)
