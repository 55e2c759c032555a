"""CPU checks of the C ABI: libshm.so builds (nvcc cross-compiles sm_103a), loads without a GPU,
exports every function include/shm.h declares, and its host-only entry points and argument
validation work without touching the device.  Also checks that the CUDA path and the oracle
stay separate (neither imports the other)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_20063_gb300 import build as B
    B.build()
    import paper_2602_20063_gb300 as S
    return S.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "shm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(shm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("shm_build_lut", "shm_query", "shm_query_backward", "shm_raycast"):
        assert must in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_helpers(lib):
    assert lib.shm_version() == 1
    assert lib.shm_records_per_glyph(32, 0) == 6 * 34 * 34
    assert lib.shm_records_per_glyph(32, 1) == 6 * 33 * 33
    assert lib.shm_records_per_glyph(0, 0) == -1
    assert lib.shm_record_bytes(0, 0) == 16 and lib.shm_record_bytes(2, 0) == 8 and lib.shm_record_bytes(0, 1) == 64
    M = 4 * 6 * 34 * 34
    # full [K][M] + tf32 hi/lo [M][Kp] (bake operands) + hi/lo slabs over M rounded up to 16 (adjoint operands)
    assert lib.shm_sh_basis_bytes(32, 8) == (81 * M + 4 * M * 96) * 4
    M9 = 4 * 6 * 11 * 11
    assert lib.shm_sh_basis_bytes(9, 8) == (81 * M9 + 2 * M9 * 96 + 2 * ((M9 + 15) // 16 * 16) * 96) * 4
    assert lib.shm_sh_basis_bytes(32, 21) == -1
    Ns = (C.c_int32 * 3)(16, 32, 5)
    offs = (C.c_int64 * 3)()
    nbytes = C.c_int64()
    assert lib.shm_lut_layout(3, Ns, 0, 0, offs, C.byref(nbytes)) == 0
    assert list(offs) == [0, 6 * 18 * 18, 6 * 18 * 18 + 6 * 34 * 34]
    assert nbytes.value == (6 * 18 * 18 + 6 * 34 * 34 + 6 * 7 * 7) * 16
    bad = (C.c_int32 * 1)(0)
    assert lib.shm_lut_layout(1, bad, 0, 0, None, None) == 1
    assert lib.shm_raycast_workspace_bytes(512, 1920, 1080) > 120 * 68 * 512 * 4
    assert lib.shm_status_string(3) == b"workspace missing or too small"


def test_validation_rejects_bad_arguments_without_a_device(lib):
    from paper_2602_20063_gb300.binding import c_lut, c_source
    # NULL descriptors / pointers are rejected before any CUDA call
    assert lib.shm_query(None, 10, None, None, None, None, None, None, None, None, None, None) == 1
    L = c_lut()
    L.n_glyphs, L.dtype, L.layout, L.N_uniform, L.data = 1, 5, 0, 8, 16
    assert lib.shm_query(C.byref(L), 10, C.c_void_p(16), None, None, None, None, None, None, None, None, None) == 1
    L.dtype, L.data = 0, 8  # misaligned pool
    assert lib.shm_query(C.byref(L), 10, C.c_void_p(16), None, None, None, None, None, None, None, None, None) == 1
    L.layout, L.data = 1, 16  # cell pools need 32-byte alignment
    assert lib.shm_query(C.byref(L), 10, C.c_void_p(16), None, None, None, None, None, None, None, None, None) == 1
    L.layout, L.data = 0, 16
    assert lib.shm_query(C.byref(L), -1, C.c_void_p(16), None, None, None, None, None, None, None, None, None) == 1
    src = c_source()
    src.kind = 99
    assert lib.shm_build_lut(C.byref(L), C.byref(src), None, 0, None) == 1
    src.kind = 0  # SH without coefficients
    assert lib.shm_build_lut(C.byref(L), C.byref(src), None, 0, None) == 1
    L.N_uniform = 0  # SH on a non-uniform pool
    src.coeffs = src.basis = 16
    L.N = L.offset = 16
    assert lib.shm_build_lut(C.byref(L), C.byref(src), None, 0, None) == 2
    assert lib.shm_sh_basis(0, 4, C.c_void_p(16), None) == 1
    # L2 fetch granularity outside -1..128 bytes
    assert lib.shm_l2_fetch_granularity(129, None) == 1
    assert lib.shm_l2_fetch_granularity(-2, None) == 1


def _imports(path):
    out = []
    for dp, _, fs in os.walk(path):
        for f in fs:
            if f.endswith(".py"):
                out.append(open(os.path.join(dp, f)).read())
    return "\n".join(out)


def test_cuda_path_and_oracle_are_separate():
    pkg = _imports(os.path.join(ROOT, "paper_2602_20063_gb300"))
    assert not re.search(r"^\s*(from|import)\s+oracle\b", pkg, flags=re.M)
    imp = lambda mod: re.compile(r"^\s*(from|import)\s+" + mod + r"\b", flags=re.M)
    orc = _imports(os.path.join(ROOT, "oracle"))
    assert not imp("paper_2602_20063_gb300").search(orc)
    inputs = _imports(os.path.join(ROOT, "shm_inputs"))
    assert not imp("paper_2602_20063_gb300").search(inputs) and not imp("oracle").search(inputs)
    # no source file of one side includes a header of the other
    for dp, _, fs in os.walk(os.path.join(ROOT, "paper_2602_20063_gb300", "csrc")):
        for f in fs:
            assert not re.search(r'#include\s+".*oracle', open(os.path.join(dp, f)).read())
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h")):
            assert not re.search(r'#include\s+".*(shm\.h|csrc|shm_device)', open(os.path.join(ROOT, "oracle", f)).read())
