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


@pytest.mark.parametrize("per_pass", [0, 2])
@pytest.mark.parametrize("prec", ["f64", "f64_emu", "split_f16", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_linop_equals_assembled_product(name, prec, per_pass):
    """Same contraction, same values: the matrix-free product equals the CSR product of the assembled
    matrix in the same precision up to the order of the sums -- and, for the FP32 forms, up to the
    FP32 rounding of the two-term values on glued faces, which the assembly stores and the
    matrix-free product never forms (about 1e-8 relative)."""
    n_e, q, macro = CASES[name]()
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(n_e), q), macro, max_tiles_per_pass=per_pass)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    u = torch.tensor(np.random.default_rng(1).normal(size=plan.n_rows), device="cuda")
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, prec).double())
    y = plan.linop(plan.pullback(ctrl), u, prec)
    assert _rel(y, K @ u) <= (1e-13 if prec.startswith("f64") else 1e-7)


def test_linop_against_oracle():
    n_e, q, macro = CASES["beam3x2x2_q3"]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, table=otables.build_table(ReferenceTile(micro), q))
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    u = np.random.default_rng(2).normal(size=plan.n_rows)
    vals = prob.assemble_lookup()
    rows = np.repeat(np.arange(plan.n_rows), np.diff(prob.rowptr))
    ref = np.zeros(plan.n_rows)
    np.add.at(ref, rows, vals * u[prob.col])
    y = plan.linop(plan.pullback(torch.tensor(macro.ctrl, device="cuda")), torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


def test_linop_beam1000_full_size():
    w = synth.workload("beam1000")
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    u = torch.tensor(np.random.default_rng(3).normal(size=plan.n_rows), device="cuda")
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "f64_emu"))
    assert _rel(plan.linop(plan.pullback(ctrl), u, "f64_emu"), K @ u) <= 1e-13
