"""The adjoint kernels (u^T dK/dP u and dL/dvalues -> dL/dP) against the oracle and finite differences."""
import numpy as np
import pytest

import synth
from oracle import adjoint as oadj, loads as oloads, tables as otables
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402


def small_case(q=1, macro=None, n_e=2):
    micro = synth.micro_cross(n_e)
    macro = macro or synth.macro_twisted_beam(2, 1, 1)
    T = otables.build_table(ReferenceTile(micro), q)
    prob = Problem(micro, macro, q, table=T, structure=False)
    tab = msasm.Tables(micro, q)
    plan = msasm.Plan(tab, macro)
    return prob, tab, plan


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f64_emu", 1e-10), ("f32", 2e-5)])
def test_grad_u_matches_oracle_complex_step(prec, tol):
    prob, tab, plan = small_case()
    u = np.random.default_rng(0).normal(size=(plan.n_points, 3))
    dt = torch.float32 if prec == "f32" else torch.float64
    ctrl = torch.tensor(prob.mmap.macro.ctrl, device="cuda")
    g = plan.assemble_grad(ctrl, 1.0, 0.3, prec, u=torch.tensor(u.ravel(), dtype=dt, device="cuda")).cpu().numpy()
    ref = oadj.gradient_all(prob, u)
    err = np.abs(g - ref).max() / np.abs(ref).max()
    print(prec, err)
    assert err <= tol, err


@pytest.mark.parametrize("prec", ["f64", "f64_emu"])
def test_grad_in_passes(prec):
    """The adjoint over tile chunks (scratch for 2 tiles) agrees with the one-pass gradient."""
    micro = synth.micro_cross(2)
    macro = synth.macro_twisted_beam(3, 2, 1)
    tab = msasm.Tables(micro, 2)
    one = msasm.Plan(tab, macro)
    chunked = msasm.Plan(tab, macro, max_tiles_per_pass=2)
    u = torch.tensor(np.random.default_rng(5).normal(size=one.n_rows), device="cuda")
    ctrl = torch.tensor(macro.ctrl, device="cuda")
    g1 = one.assemble_grad(ctrl, 1.0, 0.3, prec, u=u)
    g2 = chunked.assemble_grad(ctrl, 1.0, 0.3, prec, u=u)
    assert (torch.linalg.vector_norm(g1 - g2) / torch.linalg.vector_norm(g1)).item() <= 1e-12


def test_grad_values_mode_is_the_scatter_adjoint():
    """dL/dvalues = u_row u_col gives the same gradient as the quadratic-form mode."""
    prob, tab, plan = small_case(q=2, macro=synth.macro_perturbed_cube(seed=0))
    u = torch.tensor(np.random.default_rng(1).normal(size=plan.n_rows), device="cuda")
    rowptr, col = plan.csr()
    rows = torch.repeat_interleave(torch.arange(plan.n_rows, device="cuda"), rowptr[1:] - rowptr[:-1])
    gv = u[rows] * u[col.long()]
    ctrl = torch.tensor(prob.mmap.macro.ctrl, device="cuda")
    g1 = plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=u)
    g2 = plan.assemble_grad(ctrl, 1.0, 0.3, "f64", grad_values=gv)
    assert (g1 - g2).abs().max().item() <= 1e-12 * g1.abs().max().item()


def test_autograd_function_vs_finite_differences():
    prob, tab, plan = small_case(q=2, macro=synth.macro_twisted_beam(2, 2, 1))
    ctrl = torch.tensor(prob.mmap.macro.ctrl, device="cuda", requires_grad=True)
    r = torch.tensor(np.random.default_rng(2).normal(size=plan.nnz), device="cuda")
    L = (msasm.assemble_stiffness(ctrl, plan) * r).sum()
    (g,) = torch.autograd.grad(L, ctrl)
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in rng.choice(plan.n_ctrl, 6, replace=False):
        for p in range(3):
            c = ctrl.detach().clone()
            c[k, p] += h
            lp = (plan.assemble(c) * r).sum().item()
            c[k, p] -= 2 * h
            lm = (plan.assemble(c) * r).sum().item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k, p].item()) <= 1e-6 * max(1.0, g.abs().max().item()), (k, p, fd, g[k, p].item())


def test_traction_load_and_face_points_match_oracle():
    m = synth.macro_quarter_arc(4, 2, 2)
    micro = synth.micro_cross(2)
    prob = Problem(micro, m, 1, structure=False)
    plan = msasm.Plan(msasm.Tables(micro, 1), m)
    for face in (0, 1, 4):
        assert np.array_equal(plan.face_points(face), oloads.face_points(prob, face))
        f = plan.traction_load(face, (0.2, -1.0, 0.7), m.ctrl).reshape(-1, 3)
        ref = oloads.traction_load(prob, face, (0.2, -1.0, 0.7))
        assert np.abs(f - ref).max() <= 1e-13 * np.abs(ref).max()


def cantilever_setup(nx=4, ny=4, nz=2):
    m = synth.macro_cantilever(nx, ny, nz)
    micro = synth.micro_cross(2)
    tab = msasm.Tables(micro, 3)
    plan = msasm.Plan(tab, m)
    fixed_pts = plan.face_points(0)
    fixed = torch.tensor(np.concatenate([3 * fixed_pts + a for a in range(3)]), device="cuda", dtype=torch.long)
    f = torch.tensor(plan.traction_load(1, (0.0, 0.0, -1.0), m.ctrl), device="cuda")
    return m, micro, tab, plan, fixed, f


def compliance(plan, ctrl, f, fixed, tol=1e-13):
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "f64"))
    u, it, res = msasm.cg_solve(K, f, fixed, tol=tol)
    return torch.dot(f, u).item(), u, res


def test_cantilever_compliance_gradient_fd_and_oracle():
    """Compliance C = f^T u, u = K^-1 f (clamped x = 0 face, unit traction -z on x = max):
    dC/dP = -u^T (dK/dP) u, checked by central differences (step 1e-4, re-solved) on 20 seeded
    control-point coordinates and by the oracle's complex step of u^T K u.  The step balances the
    O(h^2) truncation against the CG rounding floor (true residual ~5e-12) divided by h: on this
    problem h = 1e-6, 1e-5, 1e-4, 1e-3 give relative differences of about 6e-6, 1e-6, 1e-7, 8e-7."""
    m, micro, tab, plan, fixed, f = cantilever_setup()
    ctrl = torch.tensor(m.ctrl, device="cuda")
    C0, u, res = compliance(plan, ctrl, f, fixed)
    assert res < 1e-10          # true residual at its rounding floor (about 5e-12 here)
    g = -plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=u)
    rng = np.random.default_rng(0)
    coords = [(int(k), int(p)) for k, p in zip(rng.choice(plan.n_ctrl, 20, replace=False), rng.integers(0, 3, 20))]
    h = 1e-4
    fd = []
    for k, p in coords:
        c = ctrl.clone(); c[k, p] += h
        cp, _, _ = compliance(plan, c, f, fixed)
        c[k, p] -= 2 * h
        cm, _, _ = compliance(plan, c, f, fixed)
        fd.append((cp - cm) / (2 * h))
    fd = np.array(fd)
    gk = np.array([g[k, p].item() for k, p in coords])
    scale = np.abs(gk).max()
    print("compliance", C0, "max |fd - adj| / max|g|", np.abs(fd - gk).max() / scale)
    assert np.abs(fd - gk).max() <= 2e-6 * scale
    prob = Problem(micro, m, 3, table=otables.build_table(ReferenceTile(micro), 3), structure=False)
    cs = -oadj.gradient_complex_step(prob, u.cpu().numpy(), coords)
    assert np.abs(cs - gk).max() <= 1e-10 * scale


def test_cantilever_f32_adjoint_on_the_solved_state():
    """The FP32 adjoint on a bending state, whose large rigid-body displacement the translation-free
    blocks v = u - u_ref(t) remove before the reduced-precision contraction."""
    m, micro, tab, plan, fixed, f = cantilever_setup()
    ctrl = torch.tensor(m.ctrl, device="cuda")
    _, u, _ = compliance(plan, ctrl, f, fixed)
    g64 = plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=u)
    g32 = plan.assemble_grad(ctrl, 1.0, 0.3, "f32", u=u.float())
    err = (torch.linalg.vector_norm(g32 - g64) / torch.linalg.vector_norm(g64)).item()
    print("f32 adjoint on the cantilever state: rel err", err)
    assert err <= 1e-3


def test_cantilever2000_gradient_vs_oracle_complex_step():
    """The full cantilever (20 x 20 x 5 tiles, 1,852,800 DOFs): FP64 and FP32 adjoint gradients at the
    solved state against the oracle's complex step on 12 seeded control-point coordinates (the oracle
    sums only the tiles whose span uses the control point)."""
    m, micro, tab, plan, fixed, f = cantilever_setup(20, 20, 5)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "f64_emu"))
    u, it, res = msasm.cg_solve(K, f, fixed, tol=1e-13, max_iter=30000)
    assert res < 1e-8, (it, res)
    g64 = plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=u)
    gemu = plan.assemble_grad(ctrl, 1.0, 0.3, "f64_emu", u=u)
    g32 = plan.assemble_grad(ctrl, 1.0, 0.3, "f32", u=u.float())
    rng = np.random.default_rng(0)
    coords = [(int(k), int(p)) for k, p in zip(rng.choice(plan.n_ctrl, 12, replace=False), rng.integers(0, 3, 12))]
    prob = Problem(micro, m, 3, table=otables.build_table(ReferenceTile(micro), 3), structure=False)
    # the oracle's tile-relative form: with the plain form, its own rounding on the bending state's
    # large rigid-body displacement is about 3e-10 of the gradient
    cs = oadj.gradient_complex_step(prob, u.cpu().numpy(), coords, relative=True)
    scale = np.abs(cs).max()
    e64 = np.abs(np.array([g64[k, p].item() for k, p in coords]) - cs).max() / scale
    e32 = np.abs(np.array([g32[k, p].item() for k, p in coords]) - cs).max() / scale
    eemu = np.abs(np.array([gemu[k, p].item() for k, p in coords]) - cs).max() / scale
    rel_emu = (torch.linalg.vector_norm(gemu - g64) / torch.linalg.vector_norm(g64)).item()
    rel32 = (torch.linalg.vector_norm(g32 - g64) / torch.linalg.vector_norm(g64)).item()
    print(f"cantilever2000: CG {it} it, residual {res:.2e}; FP64 vs complex step {e64:.2e}, "
          f"FP64-accurate (tensor cores) {eemu:.2e}, FP32 {e32:.2e}; over all control points FP32 vs FP64 "
          f"{rel32:.2e}, FP64-accurate vs FP64 {rel_emu:.2e}")
    # the emulated product slices each row of G = w v_a v_b to 49 bits of its largest entry; G spans a
    # wide range within a row, so the emulated form lands near 2e-11 here (the assembly's smooth
    # coefficient rows give 1e-13)
    assert e64 <= 1e-11 and eemu <= 1e-10 and rel_emu <= 1e-10
    assert e32 <= 1e-3 and rel32 <= 1e-3
