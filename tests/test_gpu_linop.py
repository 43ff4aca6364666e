"""Matrix-free y = K u (Sec. 4.2, eq. 74) against the assembled CSR product and the oracle."""
import numpy as np
import pytest

import synth
from oracle import tables as otables
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402

CASES = {
    "cube8": lambda: (2, 2, synth.macro_perturbed_cube(seed=0)),
    "beam3x2x2_q3": lambda: (2, 3, synth.macro_twisted_beam(3, 2, 2)),
    "ragged_5x1x3_ne3_q2": lambda: (3, 2, synth.macro_twisted_beam(5, 1, 3)),
}


def _rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


# matrix-free against the CSR product of the same form: FP64 forms to the order of the sums; the
# FP32 form (blocks in scratch, FP64 products) up to the FP32 rounding of the two-term values on glued
# faces, which the assembly stores and the matrix-free product never forms (about 1e-8); the split
# forms, applied in the contraction's epilogue with FP32 products of u (rounded to FP32) and the block
# values, up to that FP32 arithmetic (about 1e-7)
LINOP_TOL = {"f64": 1e-13, "f64_emu": 1e-13, "f32": 1e-7, "split_f16": 5e-7, "split_bf16": 5e-7, "tf32x3": 5e-7}


@pytest.mark.parametrize("per_pass", [0, 2])
@pytest.mark.parametrize("prec", ["f64", "f64_emu", "split_f16", "f32", "split_bf16", "tf32x3"])
@pytest.mark.parametrize("name", list(CASES))
def test_linop_equals_assembled_product(name, prec, per_pass):
    """Same contraction, same values: the matrix-free product equals the CSR product of the assembled
    matrix in the same precision, to the tolerance of the form's arithmetic (LINOP_TOL)."""
    n_e, q, macro = CASES[name]()
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(n_e), q), macro, max_tiles_per_pass=per_pass)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    u = torch.tensor(np.random.default_rng(1).normal(size=plan.n_rows), device="cuda")
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, prec).double())
    y = plan.linop(plan.pullback(ctrl), u, prec)
    err = _rel(y, K @ u)
    print(name, prec, per_pass, err)
    assert err <= LINOP_TOL[prec], err


@pytest.mark.parametrize("prec,tol", [("split_f16", 2e-6), ("tf32x3", 3e-6)])
def test_linop_split_forms_against_oracle(prec, tol):
    """The epilogue-applied product (no tile matrix stored) against the oracle's assembled matrix:
    the split form's own error level."""
    n_e, q, macro = CASES["beam3x2x2_q3"]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, table=otables.build_table(ReferenceTile(micro), q))
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    u = np.random.default_rng(4).normal(size=plan.n_rows)
    vals = prob.assemble_lookup()
    rows = np.repeat(np.arange(plan.n_rows), np.diff(prob.rowptr))
    ref = np.zeros(plan.n_rows)
    np.add.at(ref, rows, vals * u[prob.col])
    y = plan.linop(plan.pullback(torch.tensor(macro.ctrl, device="cuda")), torch.tensor(u, device="cuda"),
                   prec).cpu().numpy()
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(prec, err)
    assert err <= tol, err


@pytest.mark.parametrize("prec", ["f64", "f64_emu"])
def test_linop_against_oracle(prec):
    """FP64 forms: the CUDA-core product through the blocks in scratch, and the FP64-accurate one applied
    in the contraction's epilogue (no tile matrix stored), both to 1e-12 of the oracle."""
    n_e, q, macro = CASES["beam3x2x2_q3"]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, table=otables.build_table(ReferenceTile(micro), q))
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    u = np.random.default_rng(2).normal(size=plan.n_rows)
    vals = prob.assemble_lookup()
    rows = np.repeat(np.arange(plan.n_rows), np.diff(prob.rowptr))
    ref = np.zeros(plan.n_rows)
    np.add.at(ref, rows, vals * u[prob.col])
    y = plan.linop(plan.pullback(torch.tensor(macro.ctrl, device="cuda")), torch.tensor(u, device="cuda"),
                   prec).cpu().numpy()
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


def test_linop_beam1000_full_size():
    w = synth.workload("beam1000")
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    u = torch.tensor(np.random.default_rng(3).normal(size=plan.n_rows), device="cuda")
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "f64_emu"))
    coef = plan.pullback(ctrl)
    assert _rel(plan.linop(coef, u, "f64_emu"), K @ u) <= 1e-13
    # the epilogue-applied split-FP16 product at full size, against the CSR product of the split-FP16
    # matrix (values in FP32, the product in FP64)
    K16 = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "split_f16").double())
    assert _rel(plan.linop(coef, u, "split_f16"), K16 @ u) <= 5e-7
