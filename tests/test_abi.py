"""The C ABI library builds, loads without a GPU, exports exactly the functions that
include/qc_eloc.h declares, and its structs have the layout the binding assumes.
Argument validation that happens before any CUDA call is exercised here too."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qc_eloc.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2506_23809_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_exports_match_header(lib):
    so, path = lib
    names = _declared()
    assert "qc_eloc_create" in names and "qc_eloc_eval" in names
    for n in names:
        assert hasattr(so, n), f"{n} declared but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r"\b(qc_\w+)$", out, flags=re.M)))
    assert exported == names


def test_checked_build_exports_the_same_abi(lib):
    """The bounds-checked testing build (QC_CHECKED) compiles from the same sources and
    exports exactly the same functions as the product library."""
    from paper_2506_23809_gb300 import build
    path = build.build(checked=True)
    assert path != lib[1]
    ctypes.CDLL(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert sorted(set(re.findall(r"\b(qc_\w+)$", out, flags=re.M))) == _declared()


def test_struct_layout_matches_binding(tmp_path):
    from paper_2506_23809_gb300 import binding as B
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "qc_eloc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(qc_eloc_summary), '
                   'offsetof(qc_eloc_summary, status), sizeof(qc_eloc_out), offsetof(qc_eloc_out, hit_signsum), '
                   'offsetof(qc_eloc_out, hit_list_cap));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(B.qc_eloc_summary), B.qc_eloc_summary.status.offset,
                    ctypes.sizeof(B.qc_eloc_out), B.qc_eloc_out.hit_signsum.offset, B.qc_eloc_out.hit_list_cap.offset]


def test_header_compiles_as_c_and_cpp(tmp_path):
    src = tmp_path / "inc.c"
    src.write_text('#include "qc_eloc.h"\nint main(void){return QC_OK;}\n')
    for comp, std in (("gcc", "-std=c99"), ("g++", "-std=c++11")):
        subprocess.run([comp, std, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-x",
                        "c" if comp == "gcc" else "c++", str(src), "-o", str(tmp_path / "a.out")], check=True)


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    so, _ = lib
    so.qc_eloc_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    so.qc_eloc_last_error.restype = ctypes.c_char_p
    so.qc_eloc_last_error.argtypes = [ctypes.c_void_p]
    buf = (ctypes.c_double * 16)()
    out = ctypes.c_void_p()
    cases = [(14, 6, 0, 0, None), (13, 6, 0, 0, buf), (130, 6, 0, 0, buf), (14, 5, 0, 0, buf),
             (14, 14, 0, 0, buf), (14, 0, 0, 0, buf), (14, 6, 7, 0, buf), (14, 6, 0, 3, buf)]
    for n_orb, n_elec, prec, mode, ptr in cases:
        st = so.qc_eloc_create(ptr, ptr, 0.0, n_orb, n_elec, prec, mode, ctypes.byref(out))
        assert st == -1, (n_orb, n_elec, prec, mode)
        assert so.qc_eloc_last_error(None)
        assert not out.value
    # NULL handle is rejected everywhere
    so.qc_eloc_eval.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    assert so.qc_eloc_eval(None, None, None, None, 0, None, None, 0, None, None) == -1
    so.qc_eloc_destroy.argtypes = [ctypes.c_void_p]
    assert so.qc_eloc_destroy(None) == 0
    # the work counters, a batch's row piece and a server option refuse a NULL object too
    so.qc_eloc_work.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    w = (ctypes.c_uint64 * 9)()
    assert so.qc_eloc_work(None, w, 9) == -1
    so.qc_batch_set_rows.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64]
    assert so.qc_batch_set_rows(None, 0, 0, 0) == -1
    so.qc_server_set_option.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
    assert so.qc_server_set_option(None, 3, 5) == -1
