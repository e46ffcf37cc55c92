"""The C ABI library loads and exports every entry point include/knng.h
declares; argument checks that return before any CUDA call.  CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "knng.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2112_06630_gb300 import build as b
    b.build()
    import paper_2112_06630_gb300 as knng
    return knng.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(knng_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_calls():
    names = declared_functions()
    for must in ("knng_build", "knng_init", "knng_iterate", "knng_get", "knng_destroy", "knng_bruteforce",
                 "knng_reorder", "knng_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert missing == []


def test_signatures_are_plain_c():
    src = open(HEADER).read()
    assert "torch" not in src and "at::" not in src and "std::" not in src
    assert 'extern "C"' in src


def test_strerror_and_version(lib):
    import paper_2112_06630_gb300 as knng
    assert knng.strerror(0) == "ok"
    assert "invalid" in knng.strerror(-1)
    assert "sm_103a" in knng.version()


@pytest.mark.parametrize("n,d,K,rho,delta", [
    (1, 4, 1, 0.5, 0.0),      # n < 2
    (10, 0, 3, 0.5, 0.0),     # d < 1
    (10, 4, 0, 0.5, 0.0),     # K < 1
    (10, 4, 10, 0.5, 0.0),    # K > n-1
    (10, 4, 3, 0.0, 0.0),     # rho <= 0
    (10, 4, 3, 1.5, 0.0),     # rho > 1
    (10, 4, 3, 0.5, -1.0),    # delta < 0
])
def test_invalid_arguments_rejected_before_any_device_work(lib, n, d, K, rho, delta):
    x = np.zeros((max(n, 1), max(d, 1)), np.float32)
    ids = np.zeros((max(n, 1), max(K, 1)), np.int32)
    dists = np.zeros((max(n, 1), max(K, 1)), np.float32)
    rc = lib.knng_build(x.ctypes.data, n, d, K, rho, delta, 5, 0, ids.ctypes.data, dists.ctypes.data)
    assert rc == -1


def test_k_above_64_unsupported(lib):
    """K <= 64 is built (two keys per lane above 32); K = 65 is refused, and
    so are K > 32 with the low-precision and heap flags, before any device
    work."""
    import paper_2112_06630_gb300 as knng
    x = np.zeros((100, 4), np.float32)
    ids = np.zeros((100, 65), np.int32)
    dists = np.zeros((100, 65), np.float32)
    assert lib.knng_build(x.ctypes.data, 100, 4, 65, 0.5, 0.0, 5, 0, ids.ctypes.data, dists.ctypes.data) == -5
    for flag in (knng.FLAG_BF16, knng.FLAG_FP8, knng.FLAG_HEAP_SAMPLING):
        assert lib.knng_build_ex(x.ctypes.data, 100, 4, 40, 0.5, 0.0, 5, 0, flag, None, ids.ctypes.data,
                                 dists.ctypes.data, None) == -5
    fn = lib.knng_bruteforce_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert fn(x.ctypes.data, 100, 4, 40, None, 0, ids.ctypes.data, dists.ctypes.data, None) == -5


def test_null_pointers_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.knng_init(ctypes.byref(h), None, 10, 4, 3, 0.5, 0.0, 0, 0, None) == -1
    assert lib.knng_iterate(None, None) == -1
    assert lib.knng_destroy(None) == 0
    # a refused call leaves no stale context behind: *out is NULL on error
    x = np.zeros((10, 4), np.float32)
    ids = np.zeros((10, 3), np.int32)
    flags = np.zeros((10, 3), np.uint8)
    for bad in [(None, ids, flags, 0), (x, None, flags, 0), (x, ids, None, 0), (x, ids, flags, -1)]:
        h = ctypes.c_void_p(0x1234)
        ptrs = [a.ctypes.data if a is not None else None for a in bad[:3]]
        assert lib.knng_init_from_graph(ctypes.byref(h), ptrs[0], 10, 4, 3, 0.5, 0.0, 0, 0, None, ptrs[1], ptrs[2],
                                        bad[3]) == -1
        assert h.value is None


def test_header_compiles_as_c11(tmp_path):
    """The header is usable from plain C: a C11 translation unit that takes
    the address of every declared call compiles without warnings."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    names = declared_functions()
    src = tmp_path / "use_knng.c"
    src.write_text('#include "knng.h"\n#include <stddef.h>\n'
                   "const void *knng_calls[] = {\n"
                   + "".join(f"    (const void *)&{n},\n" for n in names)
                   + "    NULL\n};\n")
    cuda_inc = "/usr/local/cuda/include"
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-c", str(src), "-o",
                        str(tmp_path / "use_knng.o"), f"-I{os.path.join(ROOT, 'include')}", f"-I{cuda_inc}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_descriptor_layouts_match_the_binding(tmp_path):
    """The ctypes descriptors of the binding have the C structs' size and
    field offsets (a plain C program prints them)."""
    import shutil
    import subprocess
    import paper_2112_06630_gb300 as knng
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    structs = {"knng_desc": knng.Desc, "knng_desc_ex": knng.DescEx}
    body = ""
    for cname, py in structs.items():
        body += f'    printf("{cname} size %zu\\n", sizeof({cname}));\n'
        for f, _ in py._fields_:
            body += f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));\n'
    src = tmp_path / "layout.c"
    src.write_text('#include "knng.h"\n#include <stddef.h>\n#include <stdio.h>\nint main(void) {\n' + body
                   + "    return 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", str(src), "-o", str(exe),
                        f"-I{os.path.join(ROOT, 'include')}", "-I/usr/local/cuda/include"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    want = []
    for cname, py in structs.items():
        want.append(f"{cname} size {ctypes.sizeof(py)}")
        want += [f"{cname} {f} {getattr(py, f).offset}" for f, _ in py._fields_]
    assert [g for g in got if g] == want


@pytest.mark.parametrize("field,value,code", [
    ("rho", 0.0, -1), ("rho", 1.5, -1), ("delta", -1.0, -1), ("max_iters", -1, -1), ("K", 0, -1),
    ("K", 10, -1),     # K > n - 1
    ("d", 0, -1), ("K", 65, -5),
])
def test_batched_ex_rejects_any_bad_descriptor_before_device_work(lib, field, value, code):
    """knng_build_batched_ex checks every descriptor before any work: one bad
    descriptor after a good one fails the whole call."""
    import paper_2112_06630_gb300 as knng
    x = np.zeros((10, 4), np.float32)
    ids = np.zeros((10, 40), np.int32)
    dists = np.zeros((10, 40), np.float32)
    good = dict(data=x.ctypes.data, n=10, d=4, K=3, rho=0.5, delta=0.001, max_iters=5, seed=0,
                ids=ids.ctypes.data, dists=dists.ctypes.data)
    bad = dict(good, **{field: value})
    descs = (knng.DescEx * 2)(knng.DescEx(**good), knng.DescEx(**bad))
    assert lib.knng_build_batched_ex(ctypes.addressof(descs), 2, 0, None, None) == code
