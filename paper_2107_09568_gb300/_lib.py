"""ctypes binding of include/msasm.h (argument marshalling only).

The shared library is built in-tree (``build.py``).  Loading fails loudly when
it is missing: there is no fallback implementation of any step.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

c_i32, c_i64, c_u32, c_dbl, c_vp = C.c_int32, C.c_int64, C.c_uint32, C.c_double, C.c_void_p
P = C.POINTER

OK, EINVAL, ECUDA, ENOMEM, EDEGENERATE, EUNSUPPORTED, EIO = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "EDEGENERATE", -5: "EUNSUPPORTED",
                -6: "EIO"}
PRECISIONS = {"f64": 0, "f32": 1, "split_f16": 2, "split_bf16": 3, "tf32": 4, "tf32x3": 5, "f64_emu": 6}
FLAG_CHECK_DEGENERATE = 1
FLAG_STAGE_TIMES = 2


class MicroDescC(C.Structure):
    _fields_ = [("n_patches", c_i32), ("degree", P(c_i32)), ("n_elem", P(c_i32)),
                ("box_lo", P(c_dbl)), ("box_hi", P(c_dbl))]


class MacroDescC(C.Structure):
    _fields_ = [("degree", c_i32 * 3), ("n_knots", c_i32 * 3), ("knots", P(c_dbl) * 3)]


class MsasmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "msasm_build_tables": (c_i32, [P(MicroDescC), c_i32, c_i32, c_vp, P(c_vp)]),
    "msasm_tables_info": (c_i32, [c_vp, P(c_i32), P(c_i32), P(c_i32)]),
    "msasm_build_tables_q3": (c_i32, [P(MicroDescC), P(c_i32), c_i32, c_vp, P(c_vp)]),
    "msasm_tables_degrees": (c_i32, [c_vp, P(c_i32)]),
    "msasm_projection_error_q3": (c_i32, [c_vp, c_vp, P(c_i32), c_i32, c_dbl, c_dbl, c_vp, c_vp, c_vp]),
    "msasm_tables_copy": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "msasm_tables_destroy": (None, [c_vp]),
    "msasm_tables_save": (c_i32, [c_vp, C.c_char_p, c_vp]),
    "msasm_tables_load": (c_i32, [C.c_char_p, c_vp, P(c_vp)]),
    "msasm_plan_create": (c_i32, [c_vp, P(MacroDescC), c_i32, c_vp, P(c_vp), P(c_i64), P(c_i64)]),
    "msasm_plan_info": (c_i32, [c_vp, P(c_i64), P(c_i64), P(c_i64), P(c_i64), P(c_i64)]),
    "msasm_plan_csr": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "msasm_plan_numbering": (c_i32, [c_vp, c_vp, c_vp]),
    "msasm_plan_destroy": (None, [c_vp]),
    "msasm_assemble": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_vp, c_u32, c_vp]),
    "msasm_assemble_host": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_vp, c_u32, c_vp]),
    "msasm_select_degree": (c_i32, [c_vp, c_vp, c_dbl, c_i32, c_i32, c_i32, c_dbl, c_dbl, P(c_i32), P(c_dbl), c_vp]),
    "msasm_select_degrees": (c_i32, [c_vp, c_vp, c_dbl, P(c_i32), c_i32, c_i32, c_dbl, c_dbl, P(c_i32), P(c_dbl),
                                     c_vp]),
    "msasm_plan_range": (c_i32, [c_vp, c_i64, c_i64, P(c_i64), P(c_i64), P(c_i64), P(c_i64), P(c_i64)]),
    "msasm_assemble_range": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_i64, c_i64, c_vp, c_u32, c_vp]),
    "msasm_assemble_grad_range": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "msasm_degenerate_count": (c_i32, [c_vp, P(c_i64), c_vp]),
    "msasm_pullback": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp]),
    "msasm_pullback_l2": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_vp, c_vp]),
    "msasm_contract": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_vp, c_vp]),
    "msasm_scatter": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "msasm_contract_noalloc": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "msasm_assemble_grad": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "msasm_face_points": (c_i32, [c_vp, c_i32, c_vp, P(c_i64)]),
    "msasm_traction_load": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "msasm_stage_times": (c_i32, [c_vp, P(c_dbl), P(c_i32)]),
    "msasm_load_table_copy": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "msasm_linop_apply": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "msasm_projection_error": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_dbl, c_dbl, c_vp, c_vp, c_vp]),
    "msasm_projection_error_l2": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, c_dbl, c_dbl, c_vp, c_vp, c_vp]),
    "msasm_volume": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "msasm_volume_grad": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "msasm_body_load": (c_i32, [c_vp, c_vp, c_dbl, c_dbl, c_dbl, c_vp, c_vp]),
    "msasm_traction_load_lookup": (c_i32, [c_vp, c_vp, c_i32, c_dbl, c_dbl, c_dbl, c_vp, c_vp]),
    "msasm_face_table_copy": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "msasm_mlp_create": (c_i32, [c_i32, c_i32, C.c_uint64, P(c_vp)]),
    "msasm_mlp_info": (c_i32, [c_vp, P(c_i64), P(c_i32), P(c_i32)]),
    "msasm_mlp_set_params": (c_i32, [c_vp, c_vp, c_vp]),
    "msasm_mlp_get_params": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "msasm_mlp_forward": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "msasm_mlp_forward_tc": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "msasm_mlp_loss_grad": (c_i32, [c_vp, c_vp, c_vp, c_i32, P(C.c_float), c_vp, c_vp]),
    "msasm_mlp_train": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, C.c_float, c_vp, c_vp]),
    "msasm_mlp_destroy": (None, [c_vp]),
    "msasm_surrogate_create": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_i32, c_i32, C.c_uint64, c_vp,
                                       P(c_vp)]),
    "msasm_surrogate_info": (c_i32, [c_vp, P(c_i32), P(c_i32), P(c_i32)]),
    "msasm_surrogate_train": (c_i32, [c_vp, c_i32, C.c_float, c_vp, c_vp]),
    "msasm_surrogate_mlp": (c_i32, [c_vp, P(c_vp)]),
    "msasm_surrogate_basis": (c_i32, [c_vp, c_vp, c_vp]),
    "msasm_surrogate_predict": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "msasm_lowrank_contract": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp]),
    "msasm_surrogate_assemble": (c_i32, [c_vp, c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp, c_vp]),
    "msasm_surrogate_destroy": (None, [c_vp]),
    "msasm_surrogate_save": (c_i32, [c_vp, C.c_char_p, c_vp]),
    "msasm_surrogate_load": (c_i32, [C.c_char_p, c_vp, P(c_vp)]),
    "msasm_last_error": (C.c_char_p, []),
    "msasm_version": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmsasm.so (building it first if asked); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise OSError(f"libmsasm.so is not built ({path}); run paper_2107_09568_gb300/build.py")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def check(status: int):
    if status != OK:
        raise MsasmError(status, load().msasm_last_error().decode())
