"""One mesh split into tile ranges on one GPU: msasm_assemble_range gives each range's rows bit
for bit as the whole-mesh assembly does, and the ranges' partial gradients add up to the whole
gradient (eq. 69-73 is a sum over tiles)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402
from paper_2107_09568_gb300 import slabs  # noqa: E402


def _plan(macro, n_e, q, per_pass=0):
    tab = msasm.Tables(synth.micro_cross(n_e), q)
    return tab, msasm.Plan(tab, macro, max_tiles_per_pass=per_pass)


def _check_slabs(plan, ctrl, prec, world, n_elem):
    whole = plan.assemble(ctrl, 1.0, 0.3, prec)
    rowptr, _ = plan.csr()
    v_prev, r_prev = 0, 0
    for t0, t1 in slabs.slab_ranges(plan.n_tiles, world):
        r0, r1, v0, v1, he = plan.range(t0, t1)
        assert (r0, v0) == (r_prev, v_prev)                          # ranges follow each other
        assert he == slabs.halo_end(t1, n_elem)
        assert v0 == int(rowptr[r0]) and v1 == int(rowptr[r1])
        part = plan.assemble_range(ctrl, t0, t1, 1.0, 0.3, prec)
        assert part.numel() == v1 - v0
        assert torch.equal(part, whole[v0:v1]), (prec, world, t0, t1)   # bit for bit
        r_prev, v_prev = r1, v1
    assert (r_prev, v_prev) == (plan.n_rows, plan.nnz)


@pytest.mark.parametrize("prec", ["f64_emu", "split_f16"])
def test_beam1000_two_slabs_bit_identical(prec):
    m = synth.macro_twisted_beam(10, 10, 10)
    tab, plan = _plan(m, 3, 3)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    _check_slabs(plan, ctrl, prec, 2, m.n_elem)


@pytest.mark.parametrize("prec", ["f64_emu", "f32"])
def test_long_range_with_overlapped_secondary_pass(prec):
    """A range of 640 tiles with its halo and a value window: the scatter's direct pass runs in pieces
    with the secondary pass on a second stream (512 tiles and more), as in the whole-mesh assembly
    of the 1000 tiles, and both give the same values bit for bit."""
    m = synth.macro_twisted_beam(10, 10, 10)
    tab, plan = _plan(m, 3, 3)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    whole = plan.assemble(ctrl, 1.0, 0.3, prec)
    for t0, t1 in ((0, 640), (640, 1000), (100, 900)):
        r0, r1, v0, v1, he = plan.range(t0, t1)
        part = plan.assemble_range(ctrl, t0, t1, 1.0, 0.3, prec)
        assert torch.equal(part, whole[v0:v1]), (prec, t0, t1)


@pytest.mark.parametrize("prec,per_pass,world", [("f64", 0, 3), ("f32", 2, 4), ("f64_emu", 1, 5), ("tf32x3", 3, 2)])
def test_ragged_mesh_uneven_ranges_in_passes(prec, per_pass, world):
    """Ranges that end mid-layer, scratch for fewer tiles than a range plus its halo."""
    m = synth.macro_twisted_beam(5, 1, 3)
    tab, plan = _plan(m, 3, 2, per_pass)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    _check_slabs(plan, ctrl, prec, world, m.n_elem)


def test_empty_and_invalid_ranges():
    m = synth.macro_twisted_beam(3, 2, 2)
    tab, plan = _plan(m, 2, 1)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    r0, r1, v0, v1, he = plan.range(4, 4)
    assert (r0, v0) == (r1, v1) and he == 4
    lib = msasm.load()
    import ctypes as C
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.msasm_assemble_range(plan.handle, C.c_void_p(ctrl.data_ptr()), 1.0, 0.3, 0, 5, 5,
                                  C.c_void_p(out.data_ptr()), 0, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0 and torch.count_nonzero(out) == 0                 # nothing to do, nothing written
    for t0, t1 in ((-1, 2), (3, 2), (0, plan.n_tiles + 1)):
        st = lib.msasm_assemble_range(plan.handle, C.c_void_p(ctrl.data_ptr()), 1.0, 0.3, 0, t0, t1,
                                      C.c_void_p(out.data_ptr()), 0, None)
        assert st == msasm._lib.EINVAL


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f64_emu", 1e-13), ("f32", 1e-5)])
def test_gradient_ranges_add_up(prec, tol):
    m = synth.macro_cantilever(4, 4, 2)
    tab, plan = _plan(m, 2, 3)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    u = torch.tensor(np.random.default_rng(3).normal(size=plan.n_rows), device="cuda")
    uu = u if prec in ("f64", "f64_emu") else u.float()
    whole = plan.assemble_grad(ctrl, 1.0, 0.3, prec, u=uu)
    parts = [plan.assemble_grad_range(ctrl, t0, t1, 1.0, 0.3, prec, u=uu)
             for t0, t1 in slabs.slab_ranges(plan.n_tiles, 3)]
    total = slabs.allreduce_gradient(sum(parts), None)
    err = (torch.linalg.vector_norm(total - whole) / torch.linalg.vector_norm(whole)).item()
    assert err <= tol, err
