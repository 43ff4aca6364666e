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
