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


# ---------------------------------------------------------------- L2 projection (eq. 20-24)
def _l2_block(mm, t, q, lam, mu, n_g):
    """The oracle's L2 coefficients of tile t in the pullback layout (9, 9 n_pi): [3a + b][9C + 3i + j]."""
    return oproj.l2_coefficients(mm, t, q, lam, mu, n_g).reshape(-1, 9).T


@pytest.mark.parametrize("q,n_g", [(3, 4), (3, 6), (2, 9), (0, 3)])
def test_l2_coefficients_parity(q, n_g):
    macro = synth.macro_twisted_beam(3, 2, 2)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), q), macro)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    got = plan.pullback_l2(ctrl, n_g).cpu().numpy()
    lam, mu = opb.lame(1.0, 0.3)
    mm = MacroMap(macro)
    for t in range(plan.n_tiles):
        ref = _l2_block(mm, t, q, lam, mu, n_g)
        assert np.abs(got[9 * t:9 * t + 9] - ref).max() <= 1e-13 * np.abs(ref).max(), t
    if n_g == q + 1:                               # the nodes' own rule: the interpolant
        nodal = plan.pullback(ctrl).cpu().numpy()
        assert np.abs(got - nodal).max() <= 1e-14 * np.abs(nodal).max()


def test_l2_assembly_parity():
    """K with the L2-projected field through the contraction and the scatter, against the oracle's
    lookup form (eq. 58) with the oracle's L2 coefficients."""
    from oracle.assembly import Problem, scatter_csr
    macro = synth.macro_twisted_beam(3, 2, 1)
    micro = synth.micro_cross(2)
    prob = Problem(micro, macro, 2)
    plan = msasm.Plan(msasm.Tables(micro, 2), macro)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    vals = plan.assemble_l2(ctrl, 5).cpu().numpy()
    n_nz = prob.T.shape[0]
    blocks = [(t, (prob.T.reshape(n_nz, -1) @ _l2_block(prob.mmap, t, 2, prob.lam, prob.mu, 5).T).reshape(n_nz, 3, 3))
              for t in range(plan.n_tiles)]
    ref = scatter_csr(prob.tile, prob.gmap, prob.rowptr, prob.col, blocks)
    assert np.linalg.norm(vals - ref) <= 1e-12 * np.linalg.norm(ref)
    # the projected field is another field: K differs from the interpolated one, by the projection error
    k_int = plan.assemble(ctrl).cpu().numpy()
    d = np.linalg.norm(vals - k_int) / np.linalg.norm(k_int)
    assert 1e-8 < d < 1e-2


@pytest.mark.parametrize("q,n_g", [(1, 4), (3, 6)])
def test_l2_projection_error_parity(q, n_g):
    macro = synth.macro_twisted_beam(4, 2, 2)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 2), macro)
    e, m = plan.projection_error(torch.tensor(macro.ctrl, device="cuda"), q, 5, n_gauss=n_g)
    ref, ref_max = oproj.projection_error(macro, q, n_s=5, n_gauss=n_g)
    assert np.abs(e.cpu().numpy() - ref).max() <= 1e-12
    assert abs(m.item() - ref_max) <= 1e-12


def test_l2_beam1000_sampled_tiles():
    """The full-size beam: L2 projection error (q = 3, 6-point load rule) of sampled tiles."""
    w = synth.workload("beam1000")
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    e, m = plan.projection_error(torch.tensor(w.macro.ctrl, device="cuda"), 3, 5, n_gauss=6)
    lam, mu = opb.lame(1.0, 0.3)
    mm = MacroMap(w.macro)
    for t in np.random.default_rng(1).choice(plan.n_tiles, 8, replace=False):
        assert abs(e[int(t)].item() - oproj.tile_projection_error(mm, int(t), 3, lam, mu, 5, n_gauss=6)) <= 1e-12
    assert m.item() == e.max().item()
