"""Projection error of the macro field (eq. 59) and the degree choice (eq. 65) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import projection as oproj, pullback as opb
from oracle.macro import MacroMap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402


@pytest.mark.parametrize("name,macro", [("cube8", synth.macro_perturbed_cube(seed=0)),
                                        ("beam4x2x2", synth.macro_twisted_beam(4, 2, 2)),
                                        ("arc4x2x2", synth.macro_quarter_arc(4, 2, 2))])
@pytest.mark.parametrize("q,n_s", [(0, 3), (2, 5), (3, 5), (5, 4)])
def test_projection_error_parity(name, macro, q, n_s):
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 2), macro)
    e, m = plan.projection_error(torch.tensor(macro.ctrl, device="cuda"), q, n_s)
    ref, ref_max = oproj.projection_error(macro, q, n_s=n_s)
    assert np.abs(e.cpu().numpy() - ref).max() <= 1e-12
    assert abs(m.item() - ref_max) <= 1e-12


def test_degree_selection_matches_oracle():
    macro = synth.macro_twisted_beam(4, 2, 2)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 2), macro)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    for tol in (1e-2, 1e-4, 1e-6):
        assert msasm.select_projection_degree(plan, ctrl, tol, 0, 7) == oproj.select_degree(macro, tol, 0, 7)


def test_beam1000_sampled_tiles():
    w = synth.workload("beam1000")
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    e, m = plan.projection_error(torch.tensor(w.macro.ctrl, device="cuda"), 3, 5)
    lam, mu = opb.lame(1.0, 0.3)
    mm = MacroMap(w.macro)
    for t in np.random.default_rng(0).choice(plan.n_tiles, 8, replace=False):
        assert abs(e[int(t)].item() - oproj.tile_projection_error(mm, int(t), 3, lam, mu, 5)) <= 1e-12
    assert m.item() == e.max().item()
