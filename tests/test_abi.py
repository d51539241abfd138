"""The C ABI: libvie loads, exports every symbol include/vie.h declares, and
rejects bad arguments on the host (no GPU needed for these paths)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "vie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vie_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    vie = pytest.importorskip("paper_1811_00484_gb300")
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(vie.lib, name), name
    assert sorted(vie.EXPORTS) == declared


def test_status_strings():
    vie = pytest.importorskip("paper_1811_00484_gb300")
    for code, text in vie.STATUS.items():
        assert vie.lib.vie_status_string(code).decode() == text
    assert vie.lib.vie_status_string(99).decode() == "unknown status"


@pytest.mark.parametrize("grid,tol,msg", [
    ((0, 4, 4, 5e-3, 3e8), 1e-6, "outside"),
    ((4, 4, 513, 5e-3, 3e8), 1e-6, "outside"),
    ((11, 4, 4, 5e-3, 3e8), 1e-6, "prime factor"),      # 22 = 2 * 11
    ((4, 4, 4, -1.0, 3e8), 1e-6, "voxel edge"),
    ((4, 4, 4, 5e-3, 3e8), 0.0, "tol"),
    ((4, 4, 4, 5e-3, 3e8), 1.5, "tol"),
])
def test_compress_rejects_bad_arguments_before_any_cuda_call(grid, tol, msg):
    vie = pytest.importorskip("paper_1811_00484_gb300")
    g = vie.Grid(*grid)
    h = ctypes.c_void_p()
    st = vie.lib.vie_tucker_compress(ctypes.byref(g), tol, 0, 0, None, ctypes.byref(h))
    assert st == 1
    assert msg in vie.lib.vie_last_error().decode()
    assert not h.value


def test_null_operator_is_rejected():
    vie = pytest.importorskip("paper_1811_00484_gb300")
    info = vie.OpInfo()
    assert vie.lib.vie_op_info(None, ctypes.byref(info)) == 1
    assert vie.lib.vie_matvec(None, None, None, 1, 0, 0, None) == 1
    assert vie.lib.vie_solve(None, None, None, None, 1, 0, 0, None, None, None) == 1
    vie.lib.vie_destroy(None)


def test_solve_multi_rejects_bad_problem_lists():
    vie = pytest.importorskip("paper_1811_00484_gb300")
    opts = vie.SolveOpts(1e-6, 50, 200, 1e-5, 20, 0, 1, 1, 1)
    P = ctypes.c_void_p * 2
    fake = P(ctypes.c_void_p(16), ctypes.c_void_p(16))        # the same operator twice
    bufs = P(ctypes.c_void_p(64), ctypes.c_void_p(128))
    bs = (ctypes.c_int * 2)(1, 1)
    lib = vie.lib
    assert lib.vie_solve_multi(None, bufs, bufs, bufs, bs, 2, 0, 0, ctypes.byref(opts), None, None) == 1
    assert lib.vie_solve_multi(fake, bufs, bufs, bufs, bs, 0, 0, 0, ctypes.byref(opts), None, None) == 1
    assert lib.vie_solve_multi(fake, bufs, bufs, bufs, bs, 2, 0, 0, ctypes.byref(opts), None, None) == 1
    assert "share an operator" in lib.vie_last_error().decode()


def test_struct_layouts_match_header():
    """ctypes mirrors of the header structs have the C sizes."""
    vie = pytest.importorskip("paper_1811_00484_gb300")
    assert ctypes.sizeof(vie.Grid) == 3 * 4 + 4 + 2 * 8
    assert ctypes.sizeof(vie.SolveOpts) == 8 + 4 + 4 + 8 + 5 * 4 + 4   # trailing pad to 8
    assert ctypes.sizeof(vie.SolveInfo) == 4 * 4 + 8 + 65 * 8


def test_struct_offsets_match_a_c_compile_of_the_header(tmp_path):
    """Every field offset of the ctypes mirrors equals offsetof() in a C program
    compiled against include/vie.h (gcc), so a header change cannot silently
    shift a field the binding reads."""
    import os
    import shutil
    import subprocess

    vie = pytest.importorskip("paper_1811_00484_gb300")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    mirrors = {"vie_grid": vie.Grid, "vie_op_info_t": vie.OpInfo, "vie_solve_opts": vie.SolveOpts,
               "vie_solve_info": vie.SolveInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vie.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, what, val = line.split()
        py = mirrors[cname]
        got = ctypes.sizeof(py) if what == "size" else getattr(py, what).offset
        assert got == int(val), (cname, what, got, val)


def test_cp_entry_points_reject_null_operators():
    vie = pytest.importorskip("paper_1811_00484_gb300")
    assert vie.lib.vie_tucker_cp(None, 8, 1e-9, 100, 0, None) == 1
    assert "NULL" in vie.lib.vie_last_error().decode()
    assert vie.lib.vie_cp_export(None, 0, None, None, None, None, None, None) == 1
