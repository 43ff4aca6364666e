"""The learned surrogate for graded lattices: MLP kernels against the FP64 oracle, the low-rank
contraction against the oracle, and the trained surrogate against per-width quadrature tables."""
import time

import numpy as np
import pytest

import synth
from oracle import mlp as omlp
from oracle.assembly import Problem, coefficient_block

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402

H, RANK, K = 128, 32, 576


def test_mlp_loss_and_gradient_match_oracle():
    """Same (FP16-rounded) weights and data: the GPU's FP32-accumulated loss and gradient against FP64."""
    n_out = RANK * K
    rng = synth.rng(11)
    p = (rng.normal(size=omlp.n_params(H, n_out)) * 0.1).astype(np.float32)
    x = rng.uniform(-1, 1, size=64).astype(np.float32)
    t = rng.normal(size=(64, n_out)).astype(np.float32)
    net = msasm.MLP(n_out, H, seed=1)
    net.set_params(torch.tensor(p, device="cuda"))
    loss, g = net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    p16 = p.astype(np.float16).astype(np.float64)          # the weights the GPU computes with
    L_ref, g_ref = omlp.loss_grad(p16, H, n_out, x.astype(np.float64), t.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - L_ref) <= 1e-5 * L_ref
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print("mlp grad rel err", err)
    assert err <= 1e-4
    # forward, the output layer on the CUDA cores and on the tensor cores (split FP16), against FP64
    y_ref, _ = omlp.forward(p16, H, n_out, x.astype(np.float64))
    for tc in (False, True):
        y = net.forward(torch.tensor(x, device="cuda"), tensor_cores=tc).cpu().numpy()
        assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref), tc
    # new weights replace the cached tensor-core slices of the output layer
    net.set_params(torch.tensor(0.5 * p, device="cuda"))
    y_ref2, _ = omlp.forward((0.5 * p).astype(np.float16).astype(np.float64), H, n_out, x.astype(np.float64))
    y2 = net.forward(torch.tensor(x, device="cuda"), tensor_cores=True).cpu().numpy()
    assert np.linalg.norm(y2 - y_ref2) <= 1e-5 * np.linalg.norm(y_ref2)


def test_mlp_training_fits_a_smooth_family():
    n_out = 256
    rng = synth.rng(5)
    x = np.linspace(-1, 1, 64).astype(np.float32)
    a, b = rng.normal(size=(2, n_out))
    t = (np.sin(1.3 * x[:, None] + a[None, :]) * b[None, :] * 0.5).astype(np.float32)
    net = msasm.MLP(n_out, 64, seed=2)
    xt, tt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    hist = net.train(xt, tt, 3000, lr=3e-3)
    assert hist[-1] < 1e-3 * hist[0], (hist[0], hist[-1])


def test_lowrank_contract_matches_oracle():
    rng = synth.rng(3)
    n_nz, n_tiles = 9192, 7
    U = rng.normal(size=(n_nz, RANK)).astype(np.float32)
    Vt = rng.normal(size=(n_tiles, RANK, K)).astype(np.float32)
    coef = rng.normal(size=(9 * n_tiles, K))
    nz = msasm.lowrank_contract(torch.tensor(U, device="cuda"), torch.tensor(Vt, device="cuda"),
                                torch.tensor(coef, device="cuda")).cpu().numpy()
    Z = np.einsum("trk,tak->tar", Vt.astype(np.float64), coef.reshape(n_tiles, 9, K))
    ref = np.einsum("tar,mr->tma", Z, U.astype(np.float64)).reshape(n_tiles, n_nz, 3, 3)
    assert np.linalg.norm(nz - ref) <= 1e-5 * np.linalg.norm(ref)


def _graded_setup(nx=6, ny=3, nz=3):
    m = synth.macro_quarter_arc(nx, ny, nz)
    widths = synth.width_field(m.n_elem, seed=0)
    w_train = np.sort(0.15 + 0.25 * synth.rng(0).uniform(size=64))
    return m, widths, w_train


def test_surrogate_against_per_width_quadrature_and_gain():
    """A quarter arc of 6x3x3 tiles with strut widths from the sinusoidal field in [0.15, 0.40]:
    the surrogate (trained on 64 quadrature tables) against the per-width quadrature assembly (the
    method with one table per tile, the error reference), and what it gains over the method without it:
    one table at the mean width for every tile, or the nearest of the 64 training tables."""
    m, widths, w_train = _graded_setup()
    ctrl = torch.tensor(m.ctrl, device="cuda")
    base = msasm.Tables(synth.micro_cross(3, 0.3), 3)
    plan = msasm.Plan(base, m)
    coef = plan.pullback(ctrl)                              # (9 tiles, 576) FP64
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train_tabs = [msasm.Tables(synth.micro_cross(3, w), 3) for w in w_train]
    sur = msasm.Surrogate(train_tabs, w_train, coef, rank=RANK, hidden=H, power_iters=2, seed=0)
    hist = np.concatenate([sur.train(4000, 1e-3), sur.train(3000, 3e-4), sur.train(3000, 1e-4)])
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    dw = torch.tensor(widths, device="cuda")
    k_sur = sur.assemble(plan, ctrl, dw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        sur.assemble(plan, ctrl, dw, out=k_sur)
    torch.cuda.synchronize()
    t_sur = (time.perf_counter() - t0) / 3
    # per-width quadrature: one table per tile (the error reference)
    t0 = time.perf_counter()
    nz = torch.empty((plan.n_tiles, base.n_nz, 3, 3), dtype=torch.float64, device="cuda")
    for t in range(plan.n_tiles):
        tab_t = msasm.Tables(synth.micro_cross(3, float(widths[t])), 3)
        nz[t] = tab_t.contract(coef[9 * t:9 * t + 9], "f64")[0]
    k_exact = plan.scatter(nz, "f64")
    torch.cuda.synchronize()
    t_exact = time.perf_counter() - t0
    # without the network: mean-width table, or the nearest training table per tile
    k_mean = msasm.Plan(msasm.Tables(synth.micro_cross(3, 0.275), 3), m).assemble(ctrl)
    nearest = np.abs(widths[:, None] - w_train[None, :]).argmin(1)
    for t in range(plan.n_tiles):
        nz[t] = train_tabs[nearest[t]].contract(coef[9 * t:9 * t + 9], "f64")[0]
    k_near = plan.scatter(nz, "f64")
    nrm = torch.linalg.vector_norm(k_exact)
    e_sur = (torch.linalg.vector_norm(k_sur.double() - k_exact) / nrm).item()
    e_mean = (torch.linalg.vector_norm(k_mean - k_exact) / nrm).item()
    e_near = (torch.linalg.vector_norm(k_near - k_exact) / nrm).item()
    print(f"surrogate rel err {e_sur:.3e}  mean-width table {e_mean:.3e}  nearest of 64 tables {e_near:.3e}; "
          f"loss {hist[0]:.3e} -> {hist[-1]:.3e}; fit {t_fit:.1f} s, assemble {1e3 * t_sur:.2f} ms vs per-width "
          f"quadrature {1e3 * t_exact:.1f} ms")
    assert hist[-1] < 1e-3 * hist[0]
    assert e_sur < 0.1 * e_mean                # the gain in accuracy over one table for all widths
    assert t_sur < 0.2 * t_exact               # and in time over one quadrature table per tile
    assert e_sur < 1e-2


def _per_width_assembly(plan, macro_ctrl, coef, widths, base_n_nz):
    """The method without the network: one quadrature table per tile (the error reference)."""
    nz = torch.empty((plan.n_tiles, base_n_nz, 3, 3), dtype=torch.float64, device="cuda")
    for t in range(plan.n_tiles):
        tab_t = msasm.Tables(synth.micro_cross(3, float(widths[t])), 3)
        nz[t] = tab_t.contract(coef[9 * t:9 * t + 9], "f64")[0]
    return plan.scatter(nz, "f64")


def test_surrogate_on_a_map_it_was_not_fitted_to():
    """U and the MLP are fitted on the 6x3x3 quarter arc's coefficient rows (the arc of the test above);
    the surrogate then assembles a different graded lattice -- a twisted beam of 6x3x3 tiles, whose
    pulled-back fields the fit never saw -- with two width fields.  Its error against per-width
    quadrature there is reported beside the error on the arc it was fitted to, and bounded; one
    table at the mean width, on the same beam, is the method without the network."""
    m, widths, w_train = _graded_setup()
    base = msasm.Tables(synth.micro_cross(3, 0.3), 3)
    plan_arc = msasm.Plan(base, m)
    ctrl_arc = torch.tensor(m.ctrl, device="cuda")
    coef_arc = plan_arc.pullback(ctrl_arc)
    train_tabs = [msasm.Tables(synth.micro_cross(3, w), 3) for w in w_train]
    sur = msasm.Surrogate(train_tabs, w_train, coef_arc, rank=RANK, hidden=H, power_iters=2, seed=0)
    sur.train(4000, 1e-3), sur.train(3000, 3e-4), sur.train(3000, 1e-4)
    k_exact_arc = _per_width_assembly(plan_arc, m.ctrl, coef_arc, widths, base.n_nz)
    k_sur_arc = sur.assemble(plan_arc, ctrl_arc, torch.tensor(widths, device="cuda"))
    e_fit = (torch.linalg.vector_norm(k_sur_arc.double() - k_exact_arc) / torch.linalg.vector_norm(k_exact_arc)).item()
    beam = synth.macro_twisted_beam(6, 3, 3)
    plan_b = msasm.Plan(base, beam)
    ctrl_b = torch.tensor(beam.ctrl, device="cuda")
    coef_b = plan_b.pullback(ctrl_b)
    k_mean_b = msasm.Plan(msasm.Tables(synth.micro_cross(3, 0.275), 3), beam).assemble(ctrl_b)
    for seed in (0, 1):
        wb = synth.width_field(beam.n_elem, seed=seed)
        k_exact = _per_width_assembly(plan_b, beam.ctrl, coef_b, wb, base.n_nz)
        k_sur = sur.assemble(plan_b, ctrl_b, torch.tensor(wb, device="cuda"))
        nrm = torch.linalg.vector_norm(k_exact)
        e_held = (torch.linalg.vector_norm(k_sur.double() - k_exact) / nrm).item()
        e_mean = (torch.linalg.vector_norm(k_mean_b - k_exact) / nrm).item()
        print(f"fitted on the arc: arc {e_fit:.3e}; held-out twisted beam (width seed {seed}) {e_held:.3e}; "
              f"mean-width table there {e_mean:.3e}")
        # measured 4.7e-2 on the beam (1.1e-3 on the arc it was fitted to; the mean-width table 0.137 there):
        # U is fitted to the arc's coefficient rows, so its subspace carries that map's fields
        assert e_held < 1e-1                   # bounded on a map outside the fit
        assert e_held < 0.5 * e_mean           # and still better than one table for every width
        assert e_fit < e_held                  # the fitted map is the better one
