"""The allocation-free contraction entry point, for callers that cannot let the library allocate.

It must give the same nzdata as msasm_contract (FP64) on consecutive calls that
reuse its fixed device array, and refuse requests larger than that array.
Collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402
from paper_2107_09568_gb300 import _lib  # noqa: E402

TOL_F64 = 1e-12     # the FP64 tolerance of the parity tests


def _noalloc(tab, coef, n_tiles):
    lib = msasm.load()
    out = torch.full((9 * n_tiles, tab.n_nz), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.msasm_contract_noalloc(tab.handle, C.c_void_p(coef.data_ptr()), n_tiles, C.c_void_p(out.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_contract_noalloc_matches_contract_on_consecutive_calls():
    assert torch.cuda.is_available()
    tab = msasm.Tables(synth.micro_cross(3), 3)
    rng = np.random.default_rng(5)
    n_tiles = 12
    for call in range(2):                      # two calls in a row share the fixed array
        coef = torch.tensor(rng.normal(size=(9 * n_tiles, 9 * tab.n_pi)), device="cuda")
        ref = tab.contract(coef, "f64")        # the existing entry point (allocates its scratch)
        st, out = _noalloc(tab, coef, n_tiles)
        assert st == _lib.OK, msasm.load().msasm_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= TOL_F64, (call, err)


def test_contract_noalloc_rejects_oversized_requests():
    tab = msasm.Tables(synth.micro_cross(3), 3)
    n_tiles = 21                                # 9 * 21 * 23288 * 8 bytes > 32 MiB
    coef = torch.zeros((9 * n_tiles, 9 * tab.n_pi), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(tab, coef, n_tiles)
    assert st == _lib.EINVAL
    assert b"32" in msasm.load().msasm_last_error() and b"20 tiles" in msasm.load().msasm_last_error()
