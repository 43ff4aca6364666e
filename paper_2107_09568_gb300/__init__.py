"""GB300-native multiscale lookup-table stiffness assembly (arXiv 2107.09568).

Thin Python layer over the C ABI of ``include/msasm.h``: it only marshals
arguments (torch tensors for device memory and streams).  Every step of the
assembly runs in the library's CUDA kernels; there is no Python or CPU
implementation of any step here.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib
from ._lib import MsasmError, PRECISIONS, FLAG_CHECK_DEGENERATE, check, load

__all__ = ["Tables", "Plan", "MsasmError", "PRECISIONS", "load"]


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Tables:
    """Handle of msasm_build_tables: the reference tile's lookup table (FP64, on the GPU)."""

    def __init__(self, micro, q: int, n_gauss: int = 0, stream=None):
        lib = load()
        self._keep = [np.ascontiguousarray(micro.degree, dtype=np.int32).ravel(),
                      np.ascontiguousarray(micro.n_elem, dtype=np.int32).ravel(),
                      np.ascontiguousarray(micro.box_lo, dtype=np.float64).ravel(),
                      np.ascontiguousarray(micro.box_hi, dtype=np.float64).ravel()]
        d = _lib.MicroDescC(int(micro.degree.shape[0]),
                            self._keep[0].ctypes.data_as(C.POINTER(C.c_int32)),
                            self._keep[1].ctypes.data_as(C.POINTER(C.c_int32)),
                            self._keep[2].ctypes.data_as(C.POINTER(C.c_double)),
                            self._keep[3].ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        if np.ndim(q) == 0:
            check(lib.msasm_build_tables(C.byref(d), int(q), int(n_gauss), _stream(stream), C.byref(h)))
        else:                                     # one projection degree per direction
            q3 = (C.c_int32 * 3)(*[int(v) for v in q])
            check(lib.msasm_build_tables_q3(C.byref(d), q3, int(n_gauss), _stream(stream), C.byref(h)))
        self._adopt(h)

    @classmethod
    def load_file(cls, path, stream=None):
        """Tables stored by `save` (msasm_tables_load: read back, not recomputed)."""
        h = C.c_void_p()
        check(load().msasm_tables_load(os.fsencode(path), _stream(stream), C.byref(h)))
        obj = cls.__new__(cls)
        obj._keep = []
        obj._adopt(h)
        return obj

    def save(self, path, stream=None):
        """Store the tables in a file (msasm_tables_save)."""
        check(load().msasm_tables_save(self.handle, os.fsencode(path), _stream(stream)))

    def _adopt(self, h):
        lib = load()
        self.handle = h
        n_T, n_nz, n_pi = C.c_int32(), C.c_int32(), C.c_int32()
        check(lib.msasm_tables_info(h, C.byref(n_T), C.byref(n_nz), C.byref(n_pi)))
        qd = (C.c_int32 * 3)()
        check(lib.msasm_tables_degrees(h, qd))
        self.n_T, self.n_nz, self.n_pi = n_T.value, n_nz.value, n_pi.value
        self.qd = tuple(int(v) for v in qd)         # degree per direction
        self.q = self.qd[0] if len(set(self.qd)) == 1 else self.qd

    def table(self):
        """The FP64 table as a (n_nz, n_pi, 3, 3) CUDA tensor (a copy)."""
        import torch
        out = torch.empty((self.n_nz, self.n_pi, 3, 3), dtype=torch.float64, device="cuda")
        check(load().msasm_tables_copy(self.handle, _ptr(out), None, _stream()))
        return out

    def load_table(self):
        """(F (n_T, n_pi), volume table (n_pi,)) as CUDA tensors (eq. 55 body term, eq. 18)."""
        import torch
        n_T = self.n_T
        F = torch.empty((n_T, self.n_pi), dtype=torch.float64, device="cuda")
        v = torch.empty(self.n_pi, dtype=torch.float64, device="cuda")
        check(load().msasm_load_table_copy(self.handle, _ptr(F), _ptr(v), _stream()))
        return F, v

    def pairs(self):
        out = np.empty((self.n_nz, 2), dtype=np.int32)
        check(load().msasm_tables_copy(self.handle, None, out.ctypes.data_as(C.c_void_p), None))
        return out

    def contract(self, coef, precision="f64", stream=None):
        """Step 3 only: the tile blocks of eq. 58 for FP64 coefficients (9 n_tiles, 9 n_pi), as a
        (n_tiles, n_nz, 3, 3) tensor: [t, m, a, b] = K_t[(A,a),(B,b)] of pair m = (A, B)."""
        import torch
        n_tiles = coef.shape[0] // 9
        dt = torch.float64 if precision in ("f64", "f64_emu") else torch.float32
        out = torch.empty((n_tiles, self.n_nz, 3, 3), dtype=dt, device="cuda")
        check(load().msasm_contract(self.handle, PRECISIONS[precision], _ptr(coef), n_tiles, _ptr(out),
                                    _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.msasm_tables_destroy(self.handle)
            self.handle = None


class Plan:
    """Handle of msasm_plan_create: numbering, CSR pattern and scratch for one macro mesh."""

    def __init__(self, tables: Tables, macro, max_tiles_per_pass: int = 0, stream=None):
        lib = load()
        self.tables = tables
        self._knots = [np.ascontiguousarray(k, dtype=np.float64) for k in macro.knots]
        d = _lib.MacroDescC()
        for i in range(3):
            d.degree[i] = int(macro.degree[i])
            d.n_knots[i] = len(self._knots[i])
            d.knots[i] = self._knots[i].ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        n_rows, nnz = C.c_int64(), C.c_int64()
        check(lib.msasm_plan_create(tables.handle, C.byref(d), int(max_tiles_per_pass), _stream(stream),
                                    C.byref(h), C.byref(n_rows), C.byref(nnz)))
        self.handle = h
        vals = [C.c_int64() for _ in range(5)]
        check(lib.msasm_plan_info(h, *[C.byref(v) for v in vals]))
        self.n_tiles, self.n_points, self.n_rows, self.nnz, self.n_ctrl = (v.value for v in vals)

    def csr(self, stream=None):
        import torch
        rowptr = torch.empty(self.n_rows + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        check(load().msasm_plan_csr(self.handle, _ptr(rowptr), _ptr(col), _stream(stream)))
        return rowptr, col

    def numbering(self, stream=None):
        import torch
        g = torch.empty((self.n_tiles, self.tables.n_T), dtype=torch.int32, device="cuda")
        check(load().msasm_plan_numbering(self.handle, _ptr(g), _stream(stream)))
        return g

    @staticmethod
    def value_dtype(precision):
        import torch
        return torch.float64 if precision in ("f64", "f64_emu") else torch.float32

    def assemble(self, ctrl, E=1.0, nu=0.3, precision="f64", out=None, check_degenerate=False,
                 stage_times=False, stream=None):
        """Steps 1, 3, 4: CSR values of K for the control net `ctrl` (CUDA, (n_ctrl, 3) FP64)."""
        import torch
        if out is None:
            out = torch.empty(self.nnz, dtype=self.value_dtype(precision), device="cuda")
        flags = (FLAG_CHECK_DEGENERATE if check_degenerate else 0) | (_lib.FLAG_STAGE_TIMES if stage_times else 0)
        check(load().msasm_assemble(self.handle, _ptr(ctrl), float(E), float(nu), PRECISIONS[precision],
                                    _ptr(out), flags, _stream(stream)))
        return out

    def assemble_host(self, ctrl_host, values_host, E=1.0, nu=0.3, precision="f64", stream=None):
        """Same with host buffers (copies inside the call); both are torch CPU tensors (pinned for speed)."""
        check(load().msasm_assemble_host(self.handle, C.c_void_p(ctrl_host.data_ptr()), float(E), float(nu),
                                         PRECISIONS[precision], C.c_void_p(values_host.data_ptr()), 0,
                                         _stream(stream)))
        return values_host

    def stage_times(self):
        """(ms per stage [pullback, contraction, scatter], launches per stage) of the last timed assemble."""
        ms = (C.c_double * 3)()
        ln = (C.c_int32 * 3)()
        check(load().msasm_stage_times(self.handle, ms, ln))
        return list(ms), list(ln)

    def degenerate_count(self, stream=None):
        c = C.c_int64()
        check(load().msasm_degenerate_count(self.handle, C.byref(c), _stream(stream)))
        return c.value

    def pullback(self, ctrl, E=1.0, nu=0.3, stream=None):
        """Step 1 only: (9 n_tiles, 9 n_pi) FP64 coefficients (eq. 37, 42)."""
        import torch
        out = torch.empty((9 * self.n_tiles, 9 * self.tables.n_pi), dtype=torch.float64, device="cuda")
        check(load().msasm_pullback(self.handle, _ptr(ctrl), float(E), float(nu), _ptr(out), _stream(stream)))
        return out

    def scatter(self, nz, precision="f64", stream=None):
        """Step 4 only: CSR values from the tile blocks nz (n_tiles, n_nz, 3, 3) of every tile."""
        import torch
        assert nz.is_contiguous() and nz.numel() == 9 * self.n_tiles * self.tables.n_nz
        out = torch.empty(self.nnz, dtype=self.value_dtype(precision), device="cuda")
        check(load().msasm_scatter(self.handle, PRECISIONS[precision], _ptr(nz), _ptr(out), _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.msasm_plan_destroy(self.handle)
            self.handle = None


# ---------------------------------------------------------------------------------------
# adjoint, boundary data, solve
def _plan_assemble_grad(self, ctrl, E=1.0, nu=0.3, precision="f64", u=None, grad_values=None, stream=None):
    """dL/dP (n_ctrl, 3) FP64 for L = u^T K u (u given) or from dL/dvalues (grad_values given)."""
    import torch
    out = torch.empty((self.n_ctrl, 3), dtype=torch.float64, device="cuda")
    check(load().msasm_assemble_grad(self.handle, _ptr(ctrl), float(E), float(nu), PRECISIONS[precision],
                                     _ptr(u), _ptr(grad_values), _ptr(out), _stream(stream)))
    return out


def _plan_range(self, t0, t1):
    """(row0, row1, v0, v1, halo_end) of the tile range [t0, t1): the rows and CSR values its tiles own
    and the end of the tiles whose blocks reach them."""
    out = [C.c_int64() for _ in range(5)]
    check(load().msasm_plan_range(self.handle, int(t0), int(t1), *[C.byref(v) for v in out]))
    return tuple(v.value for v in out)


def _plan_assemble_range(self, ctrl, t0, t1, E=1.0, nu=0.3, precision="f64", out=None, stage_times=False,
                         stream=None):
    """The CSR values [v0, v1) owned by tiles [t0, t1) (msasm_assemble_range)."""
    import torch
    _, _, v0, v1, _ = self.range(t0, t1)
    if out is None:
        out = torch.empty(max(v1 - v0, 1), dtype=self.value_dtype(precision), device="cuda")
    flags = _lib.FLAG_STAGE_TIMES if stage_times else 0
    check(load().msasm_assemble_range(self.handle, _ptr(ctrl), float(E), float(nu), PRECISIONS[precision], int(t0),
                                      int(t1), _ptr(out), flags, _stream(stream)))
    return out[:v1 - v0]


def _plan_assemble_grad_range(self, ctrl, t0, t1, E=1.0, nu=0.3, precision="f64", u=None, grad_values=None,
                              stream=None):
    """The part of dL/dP (n_ctrl, 3) FP64 contributed by tiles [t0, t1)."""
    import torch
    out = torch.empty((self.n_ctrl, 3), dtype=torch.float64, device="cuda")
    check(load().msasm_assemble_grad_range(self.handle, _ptr(ctrl), float(E), float(nu), PRECISIONS[precision],
                                           int(t0), int(t1), _ptr(u), _ptr(grad_values), _ptr(out), _stream(stream)))
    return out


def _plan_face_points(self, face):
    n = C.c_int64(0)
    check(load().msasm_face_points(self.handle, int(face), None, C.byref(n)))
    out = np.empty(n.value, dtype=np.int32)
    check(load().msasm_face_points(self.handle, int(face), out.ctypes.data_as(C.c_void_p), C.byref(n)))
    return out


def _plan_traction_load(self, face, traction, ctrl_host):
    """Load vector (n_rows,) FP64 (host numpy) of a uniform traction on a macro face."""
    t = np.ascontiguousarray(traction, dtype=np.float64)
    c = np.ascontiguousarray(ctrl_host, dtype=np.float64)
    f = np.zeros(self.n_rows, dtype=np.float64)
    check(load().msasm_traction_load(self.handle, int(face), t.ctypes.data_as(C.c_void_p),
                                     c.ctypes.data_as(C.c_void_p), f.ctypes.data_as(C.c_void_p)))
    return f


def _plan_volume(self, ctrl, stream=None):
    """(per-tile volumes (n_tiles,), total volume (0-d tensor)) on the GPU (eq. 17, 19)."""
    import torch
    vt = torch.empty(self.n_tiles, dtype=torch.float64, device="cuda")
    tot = torch.empty((), dtype=torch.float64, device="cuda")
    check(load().msasm_volume(self.handle, _ptr(ctrl), _ptr(vt), _ptr(tot), _stream(stream)))
    return vt, tot


def _plan_volume_grad(self, ctrl, stream=None):
    """dV/dP (n_ctrl, 3) on the GPU (eq. 66-67)."""
    import torch
    g = torch.empty((self.n_ctrl, 3), dtype=torch.float64, device="cuda")
    check(load().msasm_volume_grad(self.handle, _ptr(ctrl), _ptr(g), _stream(stream)))
    return g


def _plan_body_load(self, ctrl, b, stream=None):
    """Load vector (n_rows,) FP64 on the GPU of the constant body force b (eq. 53, F = 0 term)."""
    import torch
    f = torch.empty(self.n_rows, dtype=torch.float64, device="cuda")
    check(load().msasm_body_load(self.handle, _ptr(ctrl), float(b[0]), float(b[1]), float(b[2]), _ptr(f),
                                 _stream(stream)))
    return f


def _plan_traction_load_lookup(self, ctrl, face, traction, stream=None):
    """Load vector (n_rows,) FP64 on the GPU of a uniform traction on a macro face, through the face
    tables (eq. 53-55, F >= 1; eq. 87-88)."""
    import torch
    f = torch.empty(self.n_rows, dtype=torch.float64, device="cuda")
    check(load().msasm_traction_load_lookup(self.handle, _ptr(ctrl), int(face), float(traction[0]),
                                            float(traction[1]), float(traction[2]), _ptr(f), _stream(stream)))
    return f


def _tables_face_table(self, face, stream=None):
    """The face load table of `face` (n_T, (q_a+1)(q_b+1), a < b its in-face directions) FP64 on the GPU."""
    import torch
    ia, ib = [k for k in range(3) if k != face // 2]
    out = torch.empty((self.n_T, (self.qd[ia] + 1) * (self.qd[ib] + 1)), dtype=torch.float64, device="cuda")
    check(load().msasm_face_table_copy(self.handle, int(face), _ptr(out), _stream(stream)))
    return out


def _plan_linop(self, coef, u, precision="f64", out=None, stream=None):
    """y = K u matrix-free (eq. 74) from the coefficients of plan.pullback(ctrl)."""
    import torch
    y = torch.empty(self.n_rows, dtype=torch.float64, device="cuda") if out is None else out
    check(load().msasm_linop_apply(self.handle, _ptr(coef), PRECISIONS[precision], _ptr(u), _ptr(y),
                                   _stream(stream)))
    return y


def _plan_projection_error(self, ctrl, q, n_samples=5, E=1.0, nu=0.3, n_gauss=0, stream=None):
    """(per-tile errors (n_tiles,), E_proj) of eq. 59 for degree q: of the interpolant, or with
    n_gauss > 0 of the L2 projection (eq. 20-24, load rule of n_gauss points per direction)."""
    import torch
    e = torch.empty(self.n_tiles, dtype=torch.float64, device="cuda")
    m = torch.empty((), dtype=torch.float64, device="cuda")
    if np.ndim(q) != 0:                            # one degree per direction
        if n_gauss > 0:
            raise MsasmError(-1, "the L2 projection error takes one degree")
        q3 = (C.c_int32 * 3)(*[int(v) for v in q])
        check(load().msasm_projection_error_q3(self.handle, _ptr(ctrl), q3, int(n_samples), float(E), float(nu),
                                               _ptr(e), _ptr(m), _stream(stream)))
    elif n_gauss > 0:
        check(load().msasm_projection_error_l2(self.handle, _ptr(ctrl), int(q), int(n_gauss), int(n_samples),
                                               float(E), float(nu), _ptr(e), _ptr(m), _stream(stream)))
    else:
        check(load().msasm_projection_error(self.handle, _ptr(ctrl), int(q), int(n_samples), float(E), float(nu),
                                            _ptr(e), _ptr(m), _stream(stream)))
    return e, m


def _plan_pullback_l2(self, ctrl, n_gauss, E=1.0, nu=0.3, stream=None):
    """Step 1 with the L2 projection of eq. 20-24: (9 n_tiles, 9 n_pi) FP64 coefficients."""
    import torch
    out = torch.empty((9 * self.n_tiles, 9 * self.tables.n_pi), dtype=torch.float64, device="cuda")
    check(load().msasm_pullback_l2(self.handle, _ptr(ctrl), float(E), float(nu), int(n_gauss), _ptr(out),
                                   _stream(stream)))
    return out


def _plan_assemble_l2(self, ctrl, n_gauss, E=1.0, nu=0.3, precision="f64", stream=None):
    """K with the L2-projected macro field: msasm_pullback_l2, then the contraction and the scatter."""
    return self.scatter(self.tables.contract(self.pullback_l2(ctrl, n_gauss, E, nu, stream), precision,
                                             stream=stream), precision, stream=stream)


def select_projection_degree(plan, ctrl, tol, q0, q_max, n_samples=5, E=1.0, nu=0.3, stream=None):
    """The degree of eq. 65 (msasm_select_degree): the smallest q in [q0, q_max] with E_proj <= tol, else q_max."""
    q, e = C.c_int32(), C.c_double()
    check(load().msasm_select_degree(plan.handle, _ptr(ctrl), float(tol), int(q0), int(q_max), int(n_samples),
                                     float(E), float(nu), C.byref(q), C.byref(e), _stream(stream)))
    return q.value


def select_projection_degrees(plan, ctrl, tol, q_init, q_max=7, n_samples=5, E=1.0, nu=0.3, stream=None):
    """A degree per direction (Sec. 3.3.4; msasm_select_degrees): (degrees, E_proj)."""
    qi = (C.c_int32 * 3)(*[int(v) for v in q_init])
    qo = (C.c_int32 * 3)()
    e = C.c_double()
    check(load().msasm_select_degrees(plan.handle, _ptr(ctrl), float(tol), qi, int(q_max), int(n_samples), float(E),
                                      float(nu), qo, C.byref(e), _stream(stream)))
    return tuple(int(v) for v in qo), e.value


Plan.range = _plan_range
Plan.assemble_range = _plan_assemble_range
Plan.assemble_grad_range = _plan_assemble_grad_range
Plan.projection_error = _plan_projection_error
Plan.traction_load_lookup = _plan_traction_load_lookup
Tables.face_table = _tables_face_table
Plan.pullback_l2 = _plan_pullback_l2
Plan.assemble_l2 = _plan_assemble_l2
Plan.linop = _plan_linop
Plan.assemble_grad = _plan_assemble_grad
Plan.face_points = _plan_face_points
Plan.traction_load = _plan_traction_load
Plan.volume = _plan_volume
Plan.volume_grad = _plan_volume_grad
Plan.body_load = _plan_body_load


def _autograd_function():
    import torch

    class AssembleStiffness(torch.autograd.Function):
        """values = K(ctrl) (CSR values of the plan's pattern); backward runs msasm_assemble_grad."""

        @staticmethod
        def forward(ctx, ctrl, plan, E, nu, precision):
            vals = plan.assemble(ctrl.detach(), E, nu, precision)
            ctx.save_for_backward(ctrl)
            ctx.plan, ctx.E, ctx.nu, ctx.precision = plan, E, nu, precision
            return vals

        @staticmethod
        def backward(ctx, grad_vals):
            (ctrl,) = ctx.saved_tensors
            g = ctx.plan.assemble_grad(ctrl.detach(), ctx.E, ctx.nu, ctx.precision,
                                       grad_values=grad_vals.contiguous().to(Plan.value_dtype(ctx.precision)))
            return g.to(ctrl.dtype), None, None, None, None

    return AssembleStiffness


_ASSEMBLE_FN = None


def assemble_stiffness(ctrl, plan, E=1.0, nu=0.3, precision="f64"):
    """Differentiable K(ctrl): CSR values whose backward is the library's adjoint kernels."""
    global _ASSEMBLE_FN
    if _ASSEMBLE_FN is None:
        _ASSEMBLE_FN = _autograd_function()
    return _ASSEMBLE_FN.apply(ctrl, plan, E, nu, precision)


def csr_matrix(plan, values):
    """torch sparse CSR matrix of the plan's pattern with the given values."""
    import torch
    rowptr, col = plan.csr()
    return torch.sparse_csr_tensor(rowptr, col.long(), values, size=(plan.n_rows, plan.n_rows))


def _inverse3(B):
    """Inverses of a batch of 3x3 matrices (..., 3, 3) as adjugate / determinant (elementwise ops
    only, no linear-algebra library)."""
    import torch
    a, b, c = B[..., 0, 0], B[..., 0, 1], B[..., 0, 2]
    d, e, f = B[..., 1, 0], B[..., 1, 1], B[..., 1, 2]
    g, h, i = B[..., 2, 0], B[..., 2, 1], B[..., 2, 2]
    A, Bc, C = e * i - f * h, f * g - d * i, d * h - e * g      # cofactors of the first row
    det = a * A + b * Bc + c * C
    adj = torch.stack([torch.stack([A, c * h - b * i, b * f - c * e], -1),
                       torch.stack([Bc, a * i - c * g, c * d - a * f], -1),
                       torch.stack([C, b * g - a * h, a * e - b * d], -1)], -2)
    return adj / det[..., None, None]


def cg_solve(K, f, fixed_dofs, tol=1e-12, max_iter=20000, x0=None, replace_every=50):
    """Preconditioned conjugate gradients in PyTorch on the GPU for K u = f with u = 0 on fixed_dofs
    (rows and columns of the fixed DOFs removed by masking), optionally from x0.  The
    preconditioner inverts the 3x3 diagonal block of every point (block Jacobi for the
    interleaved DOFs 3g + a); the residual is recomputed from b - K x every `replace_every`
    iterations so that the stopping test is on the true residual, and the iteration also stops
    once that residual is below 1e-8 and has not halved over 8 such checks (its rounding floor).  Returns
    (u, iters, rel_res)."""
    import torch
    n = f.numel()
    free = torch.ones(n, dtype=f.dtype, device=f.device)
    free[fixed_dofs] = 0.0
    crow, col, val = K.crow_indices(), K.col_indices(), K.values()
    rows = torch.repeat_interleave(torch.arange(n, device=f.device), crow[1:] - crow[:-1])
    same = (col // 3) == (rows // 3)
    blocks = torch.zeros((n // 3, 3, 3), dtype=f.dtype, device=f.device)
    blocks.view(-1).index_put_(((rows[same] // 3) * 9 + (rows[same] % 3) * 3 + col[same] % 3,),
                               val[same], accumulate=True)
    fm = free.view(-1, 3)
    blocks = blocks * fm[:, :, None] * fm[:, None, :] + torch.diag_embed(1.0 - fm)   # identity on fixed DOFs
    binv = _inverse3(blocks)
    prec = lambda r: (torch.bmm(binv, r.view(-1, 3, 1)).view(-1)) * free
    A = lambda x: (K @ (x * free)) * free
    b = f * free
    bn = torch.linalg.vector_norm(b)
    x = torch.zeros_like(b) if x0 is None else x0 * free
    r = b - A(x)
    z = prec(r)
    p = z.clone()
    rz = torch.dot(r, z)
    it, best, stall = 0, float("inf"), 0
    for it in range(1, max_iter + 1):
        Ap = A(p)
        alpha = rz / torch.dot(p, Ap)
        x += alpha * p
        if it % replace_every == 0:
            r = b - A(x)
            rn = (torch.linalg.vector_norm(r) / bn).item()
            if rn < tol:
                break
            # the true residual has reached its rounding floor (about eps |K| |u| / |f|); the
            # CG residual is not monotone, so this is only checked once it is small
            best, stall = (rn, 0) if rn < 0.5 * best else (best, stall + 1)
            if stall >= 8 and rn < 1e-8:
                break
        else:
            r -= alpha * Ap
        z = prec(r)
        rz_new = torch.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, (torch.linalg.vector_norm(b - A(x)) / bn).item()


# ---------------------------------------------------------------------------------------
# learned surrogate (graded lattices)
class MLP:
    """Handle of msasm_mlp (1 -> H -> H -> n_out tanh network, FP16 weights, FP32 accumulation)."""

    def __init__(self, n_out=None, hidden=128, seed=0, handle=None, owned=True):
        lib = load()
        if handle is None:
            h = C.c_void_p()
            check(lib.msasm_mlp_create(int(n_out), int(hidden), C.c_uint64(seed), C.byref(h)))
            handle = h
        self.handle, self._owned = handle, owned
        n, o, H = C.c_int64(), C.c_int32(), C.c_int32()
        check(lib.msasm_mlp_info(self.handle, C.byref(n), C.byref(o), C.byref(H)))
        self.n_params, self.n_out, self.hidden = n.value, o.value, H.value

    def params(self, half=False):
        import torch
        if half:
            out = torch.empty(self.n_params, dtype=torch.float16, device="cuda")
            check(load().msasm_mlp_get_params(self.handle, None, _ptr(out), _stream()))
        else:
            out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
            check(load().msasm_mlp_get_params(self.handle, _ptr(out), None, _stream()))
        return out

    def set_params(self, p):
        check(load().msasm_mlp_set_params(self.handle, _ptr(p.contiguous()), _stream()))

    def forward(self, x, tensor_cores=False):
        """(B, n_out) FP32 outputs; tensor_cores: the output layer as a split-FP16 tensor-core product."""
        import torch
        y = torch.empty((x.numel(), self.n_out), dtype=torch.float32, device="cuda")
        fn = load().msasm_mlp_forward_tc if tensor_cores else load().msasm_mlp_forward
        check(fn(self.handle, _ptr(x), x.numel(), _ptr(y), _stream()))
        return y

    def loss_grad(self, x, t):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = C.c_float()
        check(load().msasm_mlp_loss_grad(self.handle, _ptr(x), _ptr(t), x.numel(), C.byref(loss), _ptr(g),
                                         _stream()))
        return loss.value, g

    def train(self, x, t, steps, lr=1e-3):
        hist = np.zeros(steps, dtype=np.float32)
        check(load().msasm_mlp_train(self.handle, _ptr(x), _ptr(t), x.numel(), int(steps), float(lr),
                                     hist.ctypes.data_as(C.c_void_p), _stream()))
        return hist

    def __del__(self):
        if self._owned and getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.msasm_mlp_destroy(self.handle)
            self.handle = None


def lowrank_contract(U, Vt, coef):
    """Low-rank eq. 58: the tile blocks (n_tiles, n_nz, 3, 3) FP32 from U (n_nz, r), Vt (n_tiles, r, K) and
    coef (9 n_tiles, K) FP64."""
    import torch
    n_tiles = coef.shape[0] // 9
    nz = torch.empty((n_tiles, U.shape[0], 3, 3), dtype=torch.float32, device="cuda")
    check(load().msasm_lowrank_contract(_ptr(U.contiguous()), U.shape[0], U.shape[1], coef.shape[1],
                                        _ptr(Vt.contiguous()), _ptr(coef), n_tiles, _ptr(nz), _stream()))
    return nz


class Surrogate:
    """Handle of msasm_surrogate: T(w) ~ U V(w)^T with V from an MLP trained on quadrature tables."""

    def __init__(self, tables, widths, coef_samples, rank=32, hidden=128, power_iters=2, seed=0, stream=None):
        lib = load()
        self._tables = list(tables)
        arr = (C.c_void_p * len(tables))(*[t.handle.value for t in tables])
        w = np.ascontiguousarray(widths, dtype=np.float64)
        h = C.c_void_p()
        check(lib.msasm_surrogate_create(arr, w.ctypes.data_as(C.c_void_p), len(tables), _ptr(coef_samples),
                                         coef_samples.shape[0], int(rank), int(hidden), int(power_iters),
                                         C.c_uint64(seed), _stream(stream), C.byref(h)))
        self._adopt(h)

    @classmethod
    def load_file(cls, path, stream=None):
        """A surrogate stored by `save` (msasm_surrogate_load), MLP and Adam state included."""
        h = C.c_void_p()
        check(load().msasm_surrogate_load(os.fsencode(path), _stream(stream), C.byref(h)))
        obj = cls.__new__(cls)
        obj._tables = []
        obj._adopt(h)
        return obj

    def save(self, path, stream=None):
        """Store the surrogate in a file (msasm_surrogate_save)."""
        check(load().msasm_surrogate_save(self.handle, os.fsencode(path), _stream(stream)))

    def _adopt(self, h):
        lib = load()
        self.handle = h
        r, K, n = C.c_int32(), C.c_int32(), C.c_int32()
        check(lib.msasm_surrogate_info(h, C.byref(r), C.byref(K), C.byref(n)))
        self.rank, self.K, self.n_nz = r.value, K.value, n.value
        m = C.c_void_p()
        check(lib.msasm_surrogate_mlp(h, C.byref(m)))
        self.mlp = MLP(handle=m, owned=False)

    def train(self, steps, lr=1e-3):
        hist = np.zeros(steps, dtype=np.float32)
        check(load().msasm_surrogate_train(self.handle, int(steps), float(lr), hist.ctypes.data_as(C.c_void_p),
                                           _stream()))
        return hist

    def basis(self):
        import torch
        U = torch.empty((self.n_nz, self.rank), dtype=torch.float32, device="cuda")
        check(load().msasm_surrogate_basis(self.handle, _ptr(U), _stream()))
        return U

    def predict(self, widths):
        import torch
        Vt = torch.empty((widths.numel(), self.rank, self.K), dtype=torch.float32, device="cuda")
        check(load().msasm_surrogate_predict(self.handle, _ptr(widths), widths.numel(), _ptr(Vt), _stream()))
        return Vt


    def assemble(self, plan, ctrl, widths, E=1.0, nu=0.3, out=None):
        import torch
        if out is None:
            out = torch.empty(plan.nnz, dtype=torch.float32, device="cuda")
        check(load().msasm_surrogate_assemble(plan.handle, self.handle, _ptr(ctrl), float(E), float(nu),
                                              _ptr(widths), _ptr(out), _stream()))
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _lib._lib is not None:
            _lib._lib.msasm_surrogate_destroy(self.handle)
            self.handle = None
