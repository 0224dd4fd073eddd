"""The C-ABI library builds, loads without a GPU and exports every symbol include/rms.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rms_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_06250_gb300.builder import build
    path = build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    import paper_1810_06250_gb300 as rms
    assert sorted(rms.EXPORTS) == declared_functions()


def test_status_strings(lib):
    lib.rms_status_string.restype = ctypes.c_char_p
    texts = [lib.rms_status_string(i).decode() for i in range(6)]
    assert texts[0] == "success" and len(set(texts)) == 6
    assert lib.rms_status_string(99).decode() == "unknown status"


def test_null_plan_is_rejected(lib):
    # pure argument checks: no device is touched
    assert lib.rms_plan_destroy(None) == 0
    assert lib.rms_rmsf(None, None, None, None, None, None) == 1
    assert lib.rms_plan_sync(None, None) == 1
    out = ctypes.c_void_p(1)
    assert lib.rms_plan_create(ctypes.byref(out), None, 4, 1, None, None, 4, 3, 0) == 1
    assert out.value is None
    # host allocator: sizes and pointers are checked before anything is mapped or registered
    ptr = ctypes.c_void_p(1)
    assert lib.rms_host_alloc(ctypes.c_int64(0), ctypes.byref(ptr)) == 1 and ptr.value is None
    assert lib.rms_host_alloc(ctypes.c_int64(-5), ctypes.byref(ptr)) == 1
    assert lib.rms_host_alloc(ctypes.c_int64(4096), None) == 1
    assert lib.rms_host_free(None, ctypes.c_int64(4096)) == 1
    assert lib.rms_host_free(ctypes.c_void_p(4096), ctypes.c_int64(0)) == 1


def test_header_is_plain_c():
    # the boundary is a C ABI: the header must compile as C99 and as C++ with no torch or CUDA types
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rms.h")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc, "-fsyntax-only", std, "-Wall", "-Werror", "-x", lang, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    code = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    for t in ("torch", "at::", "cudaStream_t", "cuda_runtime", "float2", "__half", "bfloat16"):
        assert t not in code, t
