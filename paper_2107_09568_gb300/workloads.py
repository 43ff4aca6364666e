"""Measurements of the five lattice workloads through the library (used by bench.py --report).

Every number here is measured with CUDA events on the GPU; accuracy is relative Frobenius
error against the FP64 CUDA-core form of the same workload (or, for the surrogate, against
the per-width quadrature assembly, which is that form with one table per tile).
"""
from __future__ import annotations

import time

import numpy as np


def _timed(fn, reps=3, flush=None):
    import torch
    out = fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return out, float(np.median(ts))


def rel(a, b):
    import torch
    return (torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(b.double())).item()


def precision_forms(workload, forms, flush):
    """tiles/s, stiffness GB/s and error vs the FP64 CUDA-core form for each precision form."""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    w = synth.workload(workload)
    tab = msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q)
    plan = msasm.Plan(tab, w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    ref, t_ref = _timed(lambda: plan.assemble(ctrl, 1.0, 0.3, "f64"), reps=1, flush=flush)
    res = {"tiles": plan.n_tiles, "nnz": plan.nnz,
           "f64": {"ms": t_ref, "tiles_per_s": plan.n_tiles / t_ref * 1e3, "rel_fro_vs_f64_gpu": 0.0}}
    for f in forms:
        if f == "f64":
            continue
        out = torch.empty(plan.nnz, dtype=msasm.Plan.value_dtype(f), device="cuda")
        _, ms = _timed(lambda: plan.assemble(ctrl, 1.0, 0.3, f, out=out), reps=5, flush=flush)
        plan.assemble(ctrl, 1.0, 0.3, f, out=out, stage_times=True)
        st, _ = plan.stage_times()
        res[f] = {"ms": ms, "tiles_per_s": plan.n_tiles / ms * 1e3,
                  "stiffness_gbs": plan.nnz * out.element_size() / (ms / 1e3) / 1e9,
                  "rel_fro_vs_f64_gpu": rel(out, ref),
                  "stages_ms": dict(zip(["pullback", "contraction", "scatter"], [round(x, 4) for x in st]))}
        del out
    return res


def surrogate(flush, nx=20, ny=10, nz=10, steps=(4000, 3000, 3000)):
    """Graded quarter arc: fit + train the surrogate, then compare its assembly with per-width
    quadrature (one table per tile: the method without the network) in time and accuracy."""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    m = synth.macro_quarter_arc(nx, ny, nz)
    widths = synth.width_field(m.n_elem, seed=0)
    w_train = np.sort(0.15 + 0.25 * synth.rng(0).uniform(size=64))
    ctrl = torch.tensor(m.ctrl, device="cuda")
    base = msasm.Tables(synth.micro_cross(3, 0.3), 3)
    plan = msasm.Plan(base, m)
    coef = plan.pullback(ctrl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train_tabs = [msasm.Tables(synth.micro_cross(3, float(w)), 3) for w in w_train]
    torch.cuda.synchronize()
    t_tables = time.perf_counter() - t0
    rows = torch.cat([coef[9 * t:9 * t + 9] for t in range(0, plan.n_tiles, max(1, plan.n_tiles // 16))][:16 * 9])
    t0 = time.perf_counter()
    sur = msasm.Surrogate(train_tabs, w_train, rows.contiguous(), rank=32, hidden=128, power_iters=2, seed=0)
    torch.cuda.synchronize()
    t_basis = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = np.concatenate([sur.train(steps[0], 1e-3), sur.train(steps[1], 3e-4), sur.train(steps[2], 1e-4)])
    t_train = time.perf_counter() - t0
    dw = torch.tensor(widths, device="cuda")
    k_sur, ms_sur = _timed(lambda: sur.assemble(plan, ctrl, dw), reps=5, flush=flush)
    # per-width quadrature: one table per tile (the error reference and the method without the network)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nzd = torch.empty((plan.n_tiles, base.n_nz, 3, 3), dtype=torch.float64, device="cuda")
    for t in range(plan.n_tiles):
        tab_t = msasm.Tables(synth.micro_cross(3, float(widths[t])), 3)
        nzd[t] = tab_t.contract(coef[9 * t:9 * t + 9], "f64")[0]
    k_exact = plan.scatter(nzd, "f64")
    torch.cuda.synchronize()
    ms_exact = 1e3 * (time.perf_counter() - t0)
    nearest = np.abs(widths[:, None] - w_train[None, :]).argmin(1)
    for t in range(plan.n_tiles):
        nzd[t] = train_tabs[nearest[t]].contract(coef[9 * t:9 * t + 9], "f64")[0]
    k_near = plan.scatter(nzd, "f64")
    plan_mean = msasm.Plan(msasm.Tables(synth.micro_cross(3, 0.275), 3), m)
    k_mean = plan_mean.assemble(ctrl)
    # the plain FP64 GPU form of the same mesh (one table, the mean width): CUDA-core FP64 and the
    # FP64-accurate tensor-core form
    _, ms_f64 = _timed(lambda: plan_mean.assemble(ctrl, 1.0, 0.3, "f64", out=k_mean), reps=2, flush=flush)
    k_emu = torch.empty_like(k_mean)
    _, ms_emu = _timed(lambda: plan_mean.assemble(ctrl, 1.0, 0.3, "f64_emu", out=k_emu), reps=3, flush=flush)
    del k_emu
    return {"tiles": plan.n_tiles, "nnz": plan.nnz, "rank": 32, "training_tables": 64,
            "table_build_s": t_tables, "basis_fit_s": t_basis, "train_s": t_train,
            "train_loss_first_last": [float(hist[0]), float(hist[-1])],
            "surrogate_ms": ms_sur, "surrogate_tiles_per_s": plan.n_tiles / ms_sur * 1e3,
            "per_width_quadrature_ms": ms_exact, "per_width_tiles_per_s": plan.n_tiles / ms_exact * 1e3,
            "rel_fro_surrogate_vs_per_width": rel(k_sur, k_exact),
            "rel_fro_nearest_training_table_vs_per_width": rel(k_near, k_exact),
            "rel_fro_mean_width_table_vs_per_width": rel(k_mean, k_exact),
            "fp64_gpu_one_table_ms": ms_f64, "fp64_emu_gpu_one_table_ms": ms_emu,
            "speedup_vs_fp64_gpu_one_table": ms_f64 / ms_sur}


def adjoint(flush, nx=20, ny=20, nz=5, n_check=20, h=1e-4, cg_tol=1e-13, fd_precision="f64"):
    """Cantilever compliance gradient: assembly, CG solve, adjoint kernels (FP64 and FP32) and central
    differences of u^T K(P) u at fixed u on n_check seeded control-point coordinates.  (Differences of
    the re-solved compliance are not meaningful at this size: the CG solution's rounding floor, a
    relative residual near 7e-10, moves C by more than the step changes it.)"""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    m = synth.macro_cantilever(nx, ny, nz)
    tab = msasm.Tables(synth.micro_cross(2), 3)
    plan = msasm.Plan(tab, m)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    fixed_pts = plan.face_points(0)
    fixed = torch.tensor(np.concatenate([3 * fixed_pts + a for a in range(3)]), device="cuda", dtype=torch.long)
    # the load through the face lookup tables on the GPU (eq. 53-55, 87-88), checked against the
    # direct quadrature of the traction on the strut end faces (the map is affine: equal to roundoff)
    f = plan.traction_load_lookup(ctrl, 1, (0.0, 0.0, -1.0))
    f_direct = torch.tensor(plan.traction_load(1, (0.0, 0.0, -1.0), m.ctrl), device="cuda")
    load_check = ((f - f_direct).abs().max() / f_direct.abs().max()).item()
    vals, ms_asm = _timed(lambda: plan.assemble(ctrl, 1.0, 0.3, "f64_emu"), reps=3, flush=flush)
    K = msasm.csr_matrix(plan, vals)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, iters, res = msasm.cg_solve(K, f, fixed, tol=cg_tol, max_iter=30000)
    torch.cuda.synchronize()
    t_cg = time.perf_counter() - t0
    C0 = torch.dot(f, u).item()
    g64, ms_g64 = _timed(lambda: plan.assemble_grad(ctrl, 1.0, 0.3, "f64", u=u), reps=3, flush=flush)
    g32, ms_g32 = _timed(lambda: plan.assemble_grad(ctrl, 1.0, 0.3, "f32", u=u.float()), reps=3, flush=flush)
    gemu, ms_gemu = _timed(lambda: plan.assemble_grad(ctrl, 1.0, 0.3, "f64_emu", u=u), reps=3, flush=flush)
    rng = np.random.default_rng(0)
    coords = [(int(k), int(p)) for k, p in zip(rng.choice(plan.n_ctrl, n_check, replace=False),
                                               rng.integers(0, 3, n_check))]
    quad = lambda c: torch.dot(u, msasm.csr_matrix(plan, plan.assemble(c, 1.0, 0.3, fd_precision)) @ u).item()
    fdq = []
    for k, p in coords:
        c = ctrl.clone(); c[k, p] += h
        qp = quad(c)
        c[k, p] -= 2 * h
        qm = quad(c)
        fdq.append((qp - qm) / (2 * h))
    fdq = np.array(fdq)
    gq = np.array([g64[k, p].item() for k, p in coords])
    out = {"tiles": plan.n_tiles, "nnz": plan.nnz, "dofs": plan.n_rows, "assemble_ms_f64_emu": ms_asm,
           "load": "face lookup tables", "load_rel_max_vs_direct_quadrature": load_check,
           "cg_iterations": iters, "cg_rel_residual": res, "cg_s": t_cg, "compliance": C0,
           "grad_ms_f64": ms_g64, "grad_ms_f64_emu": ms_gemu, "grad_ms_f32": ms_g32,
           "grad_rel_f32_vs_f64": (torch.linalg.vector_norm(g32 - g64) / torch.linalg.vector_norm(g64)).item(),
           "grad_rel_f64_emu_vs_f64": (torch.linalg.vector_norm(gemu - g64) / torch.linalg.vector_norm(g64)).item(),
           "fd_coords": coords, "fd_step": h, "fd_assembly_form": fd_precision, "cg_tol": cg_tol,
           "fd_quadratic_max_abs_diff_over_max_grad": float(np.abs(fdq - gq).max() / np.abs(gq).max())}
    return out


def volume(flush, workload="beam1000"):
    """Volume (eq. 17-19), its gradient (eq. 66-67) and a body-force load (eq. 53) of a workload."""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    w = synth.workload(workload)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    (vt, V), ms_v = _timed(lambda: plan.volume(ctrl), reps=5, flush=flush)
    g, ms_g = _timed(lambda: plan.volume_grad(ctrl), reps=5, flush=flush)
    f, ms_f = _timed(lambda: plan.body_load(ctrl, (0.0, 0.0, -9.81)), reps=5, flush=flush)
    # traction on the twisted end face (x = n_x) and on a twisted side face (y = max), through the
    # face tables, against the direct quadrature on the host
    trac = {}
    for face in (1, 3):
        ft, ms_t = _timed(lambda: plan.traction_load_lookup(ctrl, face, (0.0, 0.0, -1.0)), reps=5, flush=flush)
        ref = torch.tensor(plan.traction_load(face, (0.0, 0.0, -1.0), w.macro.ctrl), device="cuda")
        trac[f"face{face}"] = {"ms_incl_host_table": ms_t, "rel_max_vs_direct_quadrature":
                               ((ft - ref).abs().max() / ref.abs().max()).item()}
    return {"tiles": plan.n_tiles, "volume": V.item(), "volume_ms": ms_v, "volume_grad_ms": ms_g,
            "body_load_ms": ms_f, "traction_lookup": trac,
            "grad_translation_residual": (g.sum(dim=0).abs().max() / g.abs().max()).item(),
            "grad_euler_residual": abs((ctrl * g).sum().item() - 3 * V.item()) / V.item(),
            "load_total_residual": abs(f.sum().item() + 9.81 * V.item()) / (9.81 * V.item())}


def projection(flush, workload="beam1000"):
    """E_proj (eq. 59) of a workload for q = 0..6 (5^3 samples per tile) and the degree of eq. 65."""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    w = synth.workload(workload)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    out = {"tiles": plan.n_tiles, "samples_per_tile": 125}
    for q in range(0, 7):
        (_, m), ms = _timed(lambda: plan.projection_error(ctrl, q, 5), reps=3, flush=flush)
        out[f"E_proj_q{q}"] = m.item()
        out[f"ms_q{q}"] = ms
    out["degree_for_tol_1e-3"] = msasm.select_projection_degree(plan, ctrl, 1e-3, 0, 7)
    # the L2 projection of eq. 20-24 (load rule of q + 3 points per direction, at most 9)
    for q in range(0, 7):
        n_g = min(q + 3, 9)
        (_, m), ms = _timed(lambda: plan.projection_error(ctrl, q, 5, n_gauss=n_g), reps=3, flush=flush)
        out[f"E_proj_l2_q{q}"] = m.item()
        out[f"ms_l2_q{q}"] = ms
    out["l2_load_rule"] = "q + 3 points per direction (at most 9)"
    _, out["pullback_ms"] = _timed(lambda: plan.pullback(ctrl), reps=5, flush=flush)
    _, out["pullback_l2_ms_incl_host_tables"] = _timed(lambda: plan.pullback_l2(ctrl, w.q + 3), reps=5, flush=flush)
    k_int = plan.assemble(ctrl, 1.0, 0.3, "f64_emu")
    k_l2 = plan.assemble_l2(ctrl, w.q + 3, precision="f64_emu")
    out["rel_fro_K_l2_vs_K_interpolated"] = rel(k_l2, k_int)
    del k_l2
    # a degree per direction (Sec. 3.3.4) against one degree, for a tighter tolerance
    q3, e3 = msasm.select_projection_degrees(plan, ctrl, 1e-5, (w.q, w.q, w.q))
    out["degrees_per_direction_tol_1e-5"] = list(q3)
    out["E_proj_per_direction"] = e3
    out["degree_isotropic_tol_1e-5"] = msasm.select_projection_degree(plan, ctrl, 1e-5, 0, 7)
    tab3 = msasm.Tables(synth.micro_cross(w.n_e, w.width), q3)
    plan3 = msasm.Plan(tab3, w.macro)
    form = "f64_emu" if 9 * tab3.n_pi <= 576 else "f64"
    _, ms3 = _timed(lambda: plan3.assemble(ctrl, 1.0, 0.3, form), reps=3, flush=flush)
    out["assembly_per_direction"] = {"n_pi": tab3.n_pi, "form": form, "ms": ms3,
                                     "tiles_per_s": plan3.n_tiles / ms3 * 1e3}
    return out


def linop(flush, workload="beam1000"):
    """Matrix-free y = K u (eq. 74) against the CSR product of the assembled matrix: time per product
    and the memory each needs beyond the tables."""
    import torch
    import paper_2107_09568_gb300 as msasm
    import synth
    w = synth.workload(workload)
    plan = msasm.Plan(msasm.Tables(synth.micro_cross(w.n_e, w.width), w.q), w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    coef = plan.pullback(ctrl)
    u = torch.randn(plan.n_rows, dtype=torch.float64, device="cuda")
    out = {"tiles": plan.n_tiles, "nnz": plan.nnz,
           "csr_bytes_f64": plan.nnz * (8 + 4) + (plan.n_rows + 1) * 8,
           "linop_nzdata_scratch_bytes": 0, "coef_bytes": coef.numel() * 8,
           "tensor_core_forms": "tile blocks applied to u in the contraction's epilogue, never stored"}
    y = torch.empty_like(u)
    for prec in ("f64_emu", "split_f16", "split_bf16", "tf32x3"):
        _, ms = _timed(lambda: plan.linop(coef, u, prec, out=y), reps=5, flush=flush)
        out[f"linop_ms_{prec}"] = ms
    K = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "f64_emu"))
    yk, ms_csr = _timed(lambda: K @ u, reps=5, flush=flush)
    out["csr_spmv_ms_f64"] = ms_csr
    out["rel_linop_vs_csr_f64_emu"] = (torch.linalg.vector_norm(plan.linop(coef, u, "f64_emu") - yk)
                                       / torch.linalg.vector_norm(yk)).item()
    del K
    K16 = msasm.csr_matrix(plan, plan.assemble(ctrl, 1.0, 0.3, "split_f16").double())
    y16 = K16 @ u
    out["rel_linop_vs_csr_split_f16"] = (torch.linalg.vector_norm(plan.linop(coef, u, "split_f16") - y16)
                                         / torch.linalg.vector_norm(y16)).item()
    out["speedup_split_f16_vs_csr_product"] = ms_csr / out["linop_ms_split_f16"]
    return out

