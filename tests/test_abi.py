"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function that
include/lagwave.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lagwave.h")
LIB = os.path.join(ROOT, "paper_1005_0542_gb300", "liblagwave.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lag_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1005_0542_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 40
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1005_0542_gb300 import lagwave
    assert set(_declared()) == set(lagwave._PROTOS)


def test_status_text_without_gpu(lib):
    lib.lag_strerror.restype = ctypes.c_char_p
    assert lib.lag_strerror(-3) == b"Krylov solve did not converge within max_iter"
    lib.lag_version.restype = ctypes.c_int
    assert lib.lag_version() == 100


def test_struct_layouts_match_header(tmp_path):
    # sizes/offsets of the ABI structs as the C compiler sees them vs the ctypes binding
    from paper_1005_0542_gb300 import lagwave as L
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lagwave.h"\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(lag_grid),sizeof(lag_laguerre),sizeof(lag_solver),sizeof(lag_point),sizeof(lag_wavelet),'
                   'sizeof(lag_stats),sizeof(lag_request),sizeof(lag_result),offsetof(lag_request,t_out_host));return 0;}\n')
    exe = tmp_path / "sz"
    r = subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(t) for t in (L.lag_grid, L.lag_laguerre, L.lag_solver, L.lag_point, L.lag_wavelet,
                                       L.lag_stats, L.lag_request, L.lag_result)] + [L.lag_request.t_out_host.offset]
    assert got == want


def test_no_oracle_in_product_path():
    # the library package never imports the oracle
    pkg = os.path.join(ROOT, "paper_1005_0542_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_exact_slice_product_counts():
    # host-only: the exact-slice DST keeps the pairs i + j <= NS + 1 of NS slices per operand:
    # 7 eight-bit slices (28 pairs, exact pairs summed in K chunks of 256) while K = ceil(n/2) padded
    # to 64 is at most 1024, 9 six-bit slices (45 pairs) above, none outside 16 <= n, K <= 4224
    from paper_1005_0542_gb300 import lagwave as L
    assert [L.lag_dst_f64_slice_products(n) for n in (8, 15, 16, 255, 2048)] == [0, 0, 28, 28, 28]
    assert [L.lag_dst_f64_slice_products(n) for n in (2049, 4096, 8448)] == [45, 45, 45]
    assert L.lag_dst_f64_slice_products(8449) == 0
    assert sum(1 for i in range(1, 8) for j in range(1, 8) if i + j <= 8) == 28
    assert sum(1 for i in range(1, 10) for j in range(1, 10) if i + j <= 10) == 45
    assert 255 * 255 * 256 < 2 ** 24 < 255 * 255 * 259
