"""Volume, volume gradient and body-force load on the GPU against the oracle (Sec. 3.1, eq. 14-19;
Sec. 4.1.1, eq. 66-67; eq. 53-55)."""
import numpy as np
import pytest

import synth
from oracle import tables as otables, volume as ovol
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402


@pytest.mark.parametrize("n_e,q", [(2, 0), (2, 2), (3, 3), (2, 5)])
def test_load_and_volume_tables(n_e, q):
    micro = synth.micro_cross(n_e)
    tile = ReferenceTile(micro)
    F, v = msasm.Tables(micro, q).load_table()
    Fo, vo = otables.load_table(tile, q), otables.volume_table(tile, q)
    assert np.abs(F.cpu().numpy() - Fo).max() <= 1e-14 * np.abs(Fo).max() * 10
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-14 * np.abs(vo).max() * 10


CASES = {
    "cube8_q2": lambda: (2, 2, synth.macro_perturbed_cube(seed=0)),
    "beam3x2x2_q3": lambda: (2, 3, synth.macro_twisted_beam(3, 2, 2)),
    "arc4x2x2_q1": lambda: (3, 1, synth.macro_quarter_arc(4, 2, 2)),
}


def _case(name):
    n_e, q, macro = CASES[name]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, structure=False)
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    return prob, plan, torch.tensor(macro.ctrl, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_volume_and_body_load_parity(name):
    prob, plan, ctrl = _case(name)
    vt, V = plan.volume(ctrl)
    vt_o, V_o = ovol.volume_lookup(prob)
    assert np.abs(vt.cpu().numpy() - vt_o).max() <= 1e-13 * np.abs(vt_o).max()
    assert abs(V.item() - V_o) <= 1e-13 * V_o
    b = np.array([0.2, -1.0, 0.5])
    f = plan.body_load(ctrl, b).cpu().numpy().reshape(-1, 3)
    f_o = ovol.body_load(prob, b)
    # the plan and the oracle number the points the same way (checked bit-exact elsewhere)
    assert np.abs(f - f_o).max() <= 1e-13 * np.abs(f_o).max()
    np.testing.assert_allclose(f.sum(axis=0), b * V.item(), rtol=1e-12)


def test_volume_gradient_against_complex_step():
    n_e, q, macro = 2, 2, synth.macro_twisted_beam(2, 1, 1)
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, structure=False)
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    g = plan.volume_grad(torch.tensor(macro.ctrl, device="cuda")).cpu().numpy()
    n = macro.ctrl.shape[0]
    ref = ovol.volume_gradient_complex_step(prob, [(k, p) for k in range(n) for p in range(3)]).reshape(n, 3)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


def test_beam1000_volume_gradient_and_load_invariants():
    """Full size (1000 tiles): sampled tile volumes against the oracle, total load = b V, the gradient's
    translation and scaling invariants (sum dV/dP = 0, sum P . dV/dP = 3 V)."""
    w = synth.workload("beam1000")
    micro = synth.micro_cross(w.n_e, w.width)
    plan = msasm.Plan(msasm.Tables(micro, w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    vt, V = plan.volume(ctrl)
    prob = Problem(micro, w.macro, w.q, structure=False)
    t_h = otables.volume_table(prob.tile, w.q)
    for t in np.random.default_rng(0).choice(plan.n_tiles, 12, replace=False):
        ref = t_h @ ovol.node_abs_det(prob.mmap, int(t), w.q)
        assert abs(vt[int(t)].item() - ref) <= 1e-13 * ref
    b = (0.0, 0.0, -9.81)
    f = plan.body_load(ctrl, b).reshape(-1, 3).sum(dim=0).cpu().numpy()
    np.testing.assert_allclose(f, np.array(b) * V.item(), rtol=1e-12, atol=1e-12 * 9.81 * V.item())
    g = plan.volume_grad(ctrl)
    assert (g.sum(dim=0).abs().max() / g.abs().max()).item() <= 1e-12
    assert abs((ctrl * g).sum().item() - 3 * V.item()) <= 1e-12 * V.item()


# ---------------------------------------------------------------- traction through the face tables
@pytest.mark.parametrize("n_e,q", [(2, 0), (2, 3), (3, 2)])
def test_face_tables(n_e, q):
    micro = synth.micro_cross(n_e)
    tile = ReferenceTile(micro)
    tab = msasm.Tables(micro, q)
    for face in range(6):
        Fo = otables.face_load_table(tile, q, face)
        F = tab.face_table(face).cpu().numpy()
        assert np.abs(F - Fo).max() <= 1e-15, face


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("face", [0, 3, 5])
def test_traction_load_lookup_parity(name, face):
    from oracle import loads as oloads
    n_e, q, macro = CASES[name]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, structure=False)
    plan = msasm.Plan(msasm.Tables(micro, q), macro)
    tr = (0.3, -1.0, 0.5)
    f = plan.traction_load_lookup(torch.tensor(macro.ctrl, device="cuda"), face, tr).cpu().numpy()
    ref = oloads.traction_load_lookup(prob, face, tr, q).ravel()
    assert np.abs(f - ref).max() <= 1e-13 * np.abs(ref).max()


def test_cantilever2000_traction_lookup_equals_direct_quadrature():
    """The 20x20x5 cantilever's load (unit traction on the x = 20 face): its macro map is affine,
    so the lookup form equals the direct quadrature of the traction on the strut end faces."""
    m = synth.macro_cantilever(20, 20, 5)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 3), m)
    f = plan.traction_load_lookup(torch.tensor(m.ctrl, device="cuda"), 1, (0.0, 0.0, -1.0)).cpu().numpy()
    ref = plan.traction_load(1, (0.0, 0.0, -1.0), m.ctrl)
    assert np.abs(f - ref).max() <= 1e-13 * np.abs(ref).max()
    assert abs(f.sum() + 0.09 * 20 * 5) <= 1e-11           # total force: strut end area 0.09 per tile face
