"""The C-ABI library loads and exports every entry point declared in include/msasm.h (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np

import paper_2107_09568_gb300 as msasm
from paper_2107_09568_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "msasm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msasm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = msasm.load()
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name          # dlsym succeeds
        assert name in _lib.exported_symbols(), f"{name} has no Python binding"
    assert lib.msasm_version().startswith(b"msasm")


def test_host_side_validation_needs_no_gpu():
    lib = msasm.load()
    out = C.c_void_p()
    # NULL descriptor -> EINVAL before any CUDA call
    assert lib.msasm_build_tables(None, 3, 0, None, C.byref(out)) == _lib.EINVAL
    assert b"micro descriptor" in lib.msasm_last_error()
    assert lib.msasm_build_tables(None, 9, 0, None, C.byref(out)) == _lib.EINVAL   # q out of range
    # patch box outside [0,1]^3
    deg = np.full(3, 2, np.int32); ne = np.full(3, 2, np.int32)
    lo = np.array([0.0, 0.0, -0.1]); hi = np.array([1.0, 1.0, 1.0])
    d = _lib.MicroDescC(1, deg.ctypes.data_as(C.POINTER(C.c_int32)), ne.ctypes.data_as(C.POINTER(C.c_int32)),
                        lo.ctypes.data_as(C.POINTER(C.c_double)), hi.ctypes.data_as(C.POINTER(C.c_double)))
    assert lib.msasm_build_tables(C.byref(d), 2, 0, None, C.byref(out)) == _lib.EINVAL
    assert out.value is None
    assert lib.msasm_plan_create(None, None, 0, None, C.byref(out), None, None) == _lib.EINVAL
    assert lib.msasm_assemble(None, None, 1.0, 0.3, 0, None, 0, None) == _lib.EINVAL
    assert lib.msasm_tables_info(None, None, None, None) == _lib.EINVAL


def test_host_side_validation_of_the_later_entry_points():
    """Argument checks of the per-direction, L2-projection, face-table and tensor-core MLP calls
    return EINVAL before any CUDA call."""
    lib = msasm.load()
    out = C.c_void_p()
    bad_q = (C.c_int32 * 3)(1, 9, 1)
    assert lib.msasm_build_tables_q3(None, bad_q, 0, None, C.byref(out)) == _lib.EINVAL
    assert b"degrees" in lib.msasm_last_error()
    assert lib.msasm_build_tables_q3(None, None, 0, None, C.byref(out)) == _lib.EINVAL
    assert lib.msasm_tables_degrees(None, (C.c_int32 * 3)()) == _lib.EINVAL
    e = C.c_double()
    assert lib.msasm_projection_error_q3(None, None, (C.c_int32 * 3)(1, 2, 3), 5, 1.0, 0.3,
                                         None, C.byref(e), None) == _lib.EINVAL
    assert lib.msasm_projection_error_l2(None, None, 2, 5, 5, 1.0, 0.3, None, C.byref(e), None) == _lib.EINVAL
    assert lib.msasm_pullback_l2(None, None, 1.0, 0.3, 5, None, None) == _lib.EINVAL
    assert lib.msasm_traction_load_lookup(None, None, 1, 0.0, 0.0, -1.0, None, None) == _lib.EINVAL
    assert lib.msasm_face_table_copy(None, 0, None, None) == _lib.EINVAL
    assert lib.msasm_mlp_forward_tc(None, None, 4, None, None) == _lib.EINVAL


def test_edge_and_corner_points_are_rejected_before_any_cuda_call():
    """A solid-cube micro tile (one patch filling [0,1]^3) has control points on the tile's edges
    and corners, which three or more tiles share; the face-by-face gluing of the numbering, the
    pattern and the scatter does not cover them, so the table build refuses the tile."""
    lib = msasm.load()
    out = C.c_void_p()
    deg = np.full(3, 2, np.int32); ne = np.full(3, 2, np.int32)
    lo = np.zeros(3); hi = np.ones(3)
    d = _lib.MicroDescC(1, deg.ctypes.data_as(C.POINTER(C.c_int32)), ne.ctypes.data_as(C.POINTER(C.c_int32)),
                        lo.ctypes.data_as(C.POINTER(C.c_double)), hi.ctypes.data_as(C.POINTER(C.c_double)))
    assert lib.msasm_build_tables(C.byref(d), 2, 0, None, C.byref(out)) == _lib.EUNSUPPORTED
    assert b"edge or corner" in lib.msasm_last_error()
    assert out.value is None


def test_host_side_validation_of_the_range_and_degree_calls():
    """The tile-range and degree-selection entry points refuse NULL handles and bad arguments before
    any CUDA call."""
    lib = msasm.load()
    i64 = [C.c_int64() for _ in range(5)]
    assert lib.msasm_plan_range(None, 0, 1, *[C.byref(v) for v in i64]) == _lib.EINVAL
    assert lib.msasm_assemble_range(None, None, 1.0, 0.3, 0, 0, 1, None, 0, None) == _lib.EINVAL
    assert lib.msasm_assemble_grad_range(None, None, 1.0, 0.3, 0, 0, 1, None, None, None, None) == _lib.EINVAL
    q = C.c_int32()
    e = C.c_double()
    assert lib.msasm_select_degree(None, None, 1e-3, 0, 7, 5, 1.0, 0.3, C.byref(q), C.byref(e), None) == _lib.EINVAL
    q3 = (C.c_int32 * 3)(3, 3, 3)
    out3 = (C.c_int32 * 3)()
    assert lib.msasm_select_degrees(None, None, 1e-3, q3, 7, 5, 1.0, 0.3, out3, C.byref(e), None) == _lib.EINVAL


def _fnv1a64(data: bytes) -> int:
    """64-bit FNV-1a (offset basis 14695981039346656037, prime 1099511628211)."""
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _store_file(path, tag: bytes, payload: bytes, checksum=None, version=1):
    import struct
    h = _fnv1a64(payload) if checksum is None else checksum
    path.write_bytes(tag + struct.pack("<IIQ", version, 0x01020304, len(payload)) + payload + struct.pack("<Q", h))


def test_stored_files_are_checked_before_any_cuda_call(tmp_path):
    """msasm_tables_load / msasm_surrogate_load refuse a missing file, another kind of file, another
    format version, a truncated file, a checksum mismatch and a payload whose sizes do not fit the
    tile its descriptor builds, all with EIO and before anything is allocated on a device."""
    import struct
    lib = msasm.load()
    h = C.c_void_p()

    def status(path, fn=lib.msasm_tables_load):
        h.value = None
        st = fn(os.fsencode(path), None, C.byref(h))
        assert h.value is None
        return st

    assert status(tmp_path / "missing") == _lib.EIO
    assert lib.msasm_tables_load(None, None, C.byref(h)) == _lib.EINVAL
    # a payload with a valid micro descriptor: one quadratic patch on the box [0.25, 0.75]^3 (no
    # point on the tile's faces), 27 control points and 378 pairs
    deg, ne = np.array([2, 2, 2], np.int32), np.array([1, 1, 1], np.int32)
    lo, hi = np.full(3, 0.25), np.full(3, 0.75)
    desc = struct.pack("<i", 1) + deg.tobytes() + ne.tobytes() + lo.tobytes() + hi.tobytes()
    sizes = struct.pack("<7i", 1, 1, 1, 0, 27, 378, 8) + struct.pack("<7q", *range(7))
    good = tmp_path / "t.msasm"
    _store_file(good, b"MSASMTAB", desc + sizes + b"\0" * 64)
    assert status(good) == _lib.EIO                        # 27 points, 378 pairs: the arrays are missing
    assert b"table arrays" in lib.msasm_last_error()
    wrong = struct.pack("<7i", 1, 1, 1, 0, 28, 378, 8) + struct.pack("<7q", *range(7))
    _store_file(good, b"MSASMTAB", desc + wrong + b"\0" * 64)
    assert status(good) == _lib.EIO and b"do not match" in lib.msasm_last_error()
    _store_file(good, b"MSASMSUR", desc + sizes)
    assert status(good) == _lib.EIO and b"kind" in lib.msasm_last_error()
    _store_file(good, b"MSASMTAB", desc + sizes, version=2)
    assert status(good) == _lib.EIO and b"version" in lib.msasm_last_error()
    _store_file(good, b"MSASMTAB", desc + sizes, checksum=12345)
    assert status(good) == _lib.EIO and b"checksum" in lib.msasm_last_error()
    raw = good.read_bytes()
    good.write_bytes(raw[:-20])
    assert status(good) == _lib.EIO and b"truncated" in lib.msasm_last_error()
    _store_file(good, b"MSASMTAB", struct.pack("<i", 40))
    assert status(good) == _lib.EIO and b"patch count" in lib.msasm_last_error()
    bad_q = struct.pack("<7i", 9, 1, 1, 0, 27, 378, 8) + struct.pack("<7q", *range(7))
    _store_file(good, b"MSASMTAB", desc + bad_q + b"\0" * 64)
    assert status(good) == _lib.EIO and b"degrees" in lib.msasm_last_error()
    # surrogate files
    assert status(tmp_path / "missing", lib.msasm_surrogate_load) == _lib.EIO
    _store_file(good, b"MSASMSUR", struct.pack("<7i", 0, 576, 100, 8, 3, 3, 3))
    assert status(good, lib.msasm_surrogate_load) == _lib.EIO
    assert lib.msasm_tables_save(None, b"x", None) == _lib.EINVAL
    assert lib.msasm_surrogate_save(None, b"x", None) == _lib.EINVAL
