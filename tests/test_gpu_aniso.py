"""A projection degree per direction, Q_(q1,q2,q3) (the anisotropic space of Sec. 3.3.4), through
every GPU stage that uses the projection space, against the oracle."""
import numpy as np
import pytest

import synth
from oracle import loads as oloads, projection as oproj, tables as otables, volume as ovol
from oracle.assembly import Problem, coefficient_block
from oracle.micro import ReferenceTile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402

Q = (1, 3, 2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_tables():
    micro = synth.micro_cross(2)
    tile = ReferenceTile(micro)
    tab = msasm.Tables(micro, Q)
    assert tab.qd == Q and tab.n_pi == 24
    T = tab.table().cpu().numpy()
    To = otables.build_table(tile, Q)
    assert np.abs(T - To).max() <= 1e-14 * np.abs(To).max()
    F, v = tab.load_table()
    assert np.abs(F.cpu().numpy() - otables.load_table(tile, Q)).max() <= 1e-15
    assert np.abs(v.cpu().numpy() - otables.volume_table(tile, Q)).max() <= 1e-15
    for face in range(6):
        assert np.abs(tab.face_table(face).cpu().numpy() - otables.face_load_table(tile, Q, face)).max() <= 1e-15
    # equal degrees are the isotropic tables, bit for bit
    assert torch.equal(msasm.Tables(micro, (2, 2, 2)).table(), msasm.Tables(micro, 2).table())


@pytest.fixture(scope="module")
def beam():
    micro = synth.micro_cross(2)
    macro = synth.macro_twisted_beam(3, 2, 2)
    prob = Problem(micro, macro, Q)
    plan = msasm.Plan(msasm.Tables(micro, Q), macro)
    return prob, plan, torch.tensor(macro.ctrl, device="cuda")


def test_pullback_and_assembly(beam):
    prob, plan, ctrl = beam
    coef = plan.pullback(ctrl).cpu().numpy()
    for t in range(plan.n_tiles):
        ref = coefficient_block(prob.mmap, t, Q, prob.lam, prob.mu).T
        assert np.abs(coef[9 * t:9 * t + 9] - ref).max() <= 1e-13 * np.abs(ref).max()
    ref = prob.assemble_lookup()
    for prec, tol in (("f64", 1e-12), ("f64_emu", 1e-12), ("split_f16", 1e-5)):
        assert rel(plan.assemble(ctrl, 1.0, 0.3, prec).double().cpu().numpy(), ref) <= tol, prec


def test_volume_loads_and_l2(beam):
    prob, plan, ctrl = beam
    vt, V = plan.volume(ctrl)
    vo, Vo = ovol.volume_lookup(prob)
    assert np.abs(vt.cpu().numpy() - vo).max() <= 1e-13 * np.abs(vo).max()
    f = plan.body_load(ctrl, (0.0, 0.0, -1.0)).cpu().numpy()
    assert np.abs(f - ovol.body_load(prob, (0.0, 0.0, -1.0)).ravel()).max() <= 1e-13 * np.abs(f).max()
    for face in (1, 2, 5):
        ft = plan.traction_load_lookup(ctrl, face, (0.3, -1.0, 0.5)).cpu().numpy()
        ref = oloads.traction_load_lookup(prob, face, (0.3, -1.0, 0.5), Q).ravel()
        assert np.abs(ft - ref).max() <= 1e-13 * np.abs(ref).max()
    a = plan.pullback_l2(ctrl, 5).cpu().numpy()
    for t in (0, 5, 11):
        ref = oproj.l2_coefficients(prob.mmap, t, Q, prob.lam, prob.mu, 5).reshape(-1, 9).T
        assert np.abs(a[9 * t:9 * t + 9] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_adjoint_gradient(beam):
    from oracle import adjoint as oadj
    prob, plan, ctrl = beam
    u = np.random.default_rng(2).standard_normal(plan.n_rows)
    g = plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=torch.tensor(u, device="cuda")).cpu().numpy()
    coords = [(5, 0), (17, 2), (40, 1)]
    ref = oadj.gradient_complex_step(prob, u.reshape(-1, 3), coords)
    got = np.array([g[k, p] for k, p in coords])
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(g).max()


@pytest.mark.parametrize("q", [(0, 1, 2), (3, 1, 1), (2, 4, 3)])
def test_projection_error(q):
    macro = synth.macro_twisted_beam(4, 2, 2)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 2), macro)
    e, m = plan.projection_error(torch.tensor(macro.ctrl, device="cuda"), q, 5)
    ref, ref_max = oproj.projection_error(macro, q, n_s=5)
    assert np.abs(e.cpu().numpy() - ref).max() <= 1e-12 and abs(m.item() - ref_max) <= 1e-12


def test_degree_selection_per_direction():
    macro = synth.macro_twisted_beam(4, 2, 2)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(2), 2), macro)
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    for tol in (1e-3, 1e-5):
        q, err = msasm.select_projection_degrees(plan, ctrl, tol, (3, 3, 3))
        qo, erro = oproj.select_degrees(macro, tol, (3, 3, 3))
        assert q == qo and abs(err - erro) <= 1e-12
