"""The allocation-free contraction entry point, for callers that cannot let the library allocate.

It must give the nzdata of eq. 58 -- checked against the oracle's table contracted on the host in
FP64, and against msasm_contract (FP64), the entry point that allocates -- on consecutive calls that
reuse its fixed device array, and refuse requests larger than that array.
Collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import tables as otables
from oracle.micro import ReferenceTile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402
from paper_2107_09568_gb300 import _lib  # noqa: E402

TOL_F64 = 1e-12     # the FP64 tolerance of the parity tests


def _noalloc(tab, coef, n_tiles):
    lib = msasm.load()
    out = torch.full((n_tiles, tab.n_nz, 3, 3), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.msasm_contract_noalloc(tab.handle, C.c_void_p(coef.data_ptr()), n_tiles, C.c_void_p(out.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_contract_noalloc_matches_oracle_and_contract_on_consecutive_calls():
    assert torch.cuda.is_available()
    tab = msasm.Tables(synth.micro_cross(3), 3)
    T = otables.build_table(ReferenceTile(synth.micro_cross(3)), 3).reshape(tab.n_nz, -1)   # oracle, FP64
    rng = np.random.default_rng(5)
    n_tiles = 12
    for call in range(2):                      # two calls in a row share the fixed array
        coef_h = rng.normal(size=(9 * n_tiles, 9 * tab.n_pi))
        coef = torch.tensor(coef_h, device="cuda")
        st, out = _noalloc(tab, coef, n_tiles)
        assert st == _lib.OK, msasm.load().msasm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()                # tile blocks [t, m, a, b]
        want = (coef_h @ T.T).reshape(n_tiles, 3, 3, tab.n_nz).transpose(0, 3, 1, 2)   # eq. 58 on the host
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= TOL_F64, (call, err)
        ref = tab.contract(coef, "f64").cpu().numpy()   # the existing entry point (allocates its scratch)
        err_c = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err_c <= TOL_F64, (call, err_c)


def test_contract_noalloc_rejects_oversized_requests():
    tab = msasm.Tables(synth.micro_cross(3), 3)
    n_tiles = 21                                # 9 * 21 * 23288 * 8 bytes > 32 MiB
    coef = torch.zeros((9 * n_tiles, 9 * tab.n_pi), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(tab, coef, n_tiles)
    assert st == _lib.EINVAL
    assert b"32" in msasm.load().msasm_last_error() and b"20 tiles" in msasm.load().msasm_last_error()
    # a tile count whose scratch size would wrap around a 64-bit product is refused the same way
    lib = msasm.load()
    st = lib.msasm_contract_noalloc(tab.handle, C.c_void_p(coef.data_ptr()), 2 ** 61, C.c_void_p(coef.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.EINVAL
    assert b"20 tiles" in lib.msasm_last_error()
