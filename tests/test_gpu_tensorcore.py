"""Tensor-core contraction forms (tcgen05, TMEM, TMA) against the FP64 oracle.

Split FP16 (hi/lo with a 2^11-scaled low part and per-row power-of-two scales) is the
precision form held to the 1e-6 relative Frobenius error on the assembled matrices.
The other forms are reported with bounds that follow from their arithmetic: TF32x3 has
the same 22-bit operands but twice as many FP32 accumulation steps (K = 8 per MMA
instead of 16), measured 1.2e-6 on the 4000-tile beam (bound 2e-6); split BF16 keeps
16 significant bits (~4e-6, bound 3e-5); plain TF32 keeps 11 bits (~3e-4, bound 2e-3).  The stage tests feed random normal coefficients, whose dot
products cancel far more than the method's data (|result| ~ sqrt(K) |a||b| instead of
~K |a||b|), so their bound for the 1e-6 forms is 2e-6.
"""
import numpy as np
import pytest

import synth
from oracle import tables as otables
from oracle.assembly import Problem, point_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402

TOL = {"split_f16": 1e-6, "tf32x3": 2e-6, "split_bf16": 3e-5, "tf32": 2e-3, "f32": 1e-6}
TOL_RANDOM = {"split_f16": 2e-6, "tf32x3": 2e-6, "split_bf16": 3e-5, "tf32": 2e-3}
_T = {}


def oracle_table(n_e, q):
    if (n_e, q) not in _T:
        from oracle.micro import ReferenceTile
        _T[(n_e, q)] = otables.build_table(ReferenceTile(synth.micro_cross(n_e)), q)
    return _T[(n_e, q)]



def blocks_to_rows(nz):
    """The library's tile blocks (n_tiles, n_nz, 3, 3) as the rows nz[9t + 3a + b][m] of coef @ T^T."""
    t, m = nz.shape[:2]
    return nz.reshape(t, m, 9).transpose(0, 2, 1).reshape(9 * t, m)

def rel_fro(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["tf32", "split_bf16", "split_f16", "tf32x3"])
def test_tc_single_tile_small_table(prec):
    """One coefficient tile (N = 9), K = 72 (q = 1): two k-blocks, ragged m and n."""
    tab = msasm.Tables(synth.micro_cross(2), 1)
    coef = np.random.default_rng(1).normal(size=(9, 9 * tab.n_pi))
    nz = blocks_to_rows(tab.contract(torch.tensor(coef, device="cuda"), prec).cpu().numpy())
    ref = coef @ oracle_table(2, 1).reshape(tab.n_nz, -1).T
    err = rel_fro(nz, ref)
    print(prec, err)
    assert err <= TOL_RANDOM[prec], err


@pytest.mark.parametrize("prec", ["tf32", "split_bf16", "split_f16", "tf32x3"])
@pytest.mark.parametrize("n_e,q,n_tiles", [(3, 3, 61), (2, 2, 8), (2, 0, 3)])
def test_tc_contract_parity(prec, n_e, q, n_tiles):
    tab = msasm.Tables(synth.micro_cross(n_e), q)
    coef = np.random.default_rng(2).normal(size=(9 * n_tiles, 9 * tab.n_pi))
    nz = blocks_to_rows(tab.contract(torch.tensor(coef, device="cuda"), prec).cpu().numpy())
    ref = coef @ oracle_table(n_e, q).reshape(tab.n_nz, -1).T
    err = rel_fro(nz, ref)
    print(prec, n_e, q, n_tiles, err)
    assert err <= TOL_RANDOM[prec], err


@pytest.mark.parametrize("prec", ["split_f16", "tf32x3", "split_bf16", "tf32"])
def test_tc_assemble_parity(prec):
    w = synth.workload("cube8")
    micro = synth.micro_cross(2)
    prob = Problem(micro, w.macro, 2, table=oracle_table(2, 2))
    tab = msasm.Tables(micro, 2)
    plan = msasm.Plan(tab, w.macro)
    vals = plan.assemble(torch.tensor(w.macro.ctrl, device="cuda"), 1.0, 0.3, prec, check_degenerate=True)
    err = rel_fro(vals.cpu().numpy(), prob.assemble_lookup())
    print(prec, err)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["split_f16", "tf32x3", "split_bf16", "tf32", "f32"])
def test_beam4000_full_size_sampled(prec):
    """The 40x10x10 twisted beam (precision-form workload, 4000 tiles in one pass): sampled rows
    against the oracle, and the translation null space of the whole matrix."""
    w = synth.workload("beam4000")
    micro = synth.micro_cross(3)
    prob = Problem(micro, w.macro, 3, table=oracle_table(3, 3), structure=False)
    tab = msasm.Tables(micro, 3)
    plan = msasm.Plan(tab, w.macro)
    assert plan.nnz == 1614428100
    vals = plan.assemble(torch.tensor(w.macro.ctrl, device="cuda"), 1.0, 0.3, prec, check_degenerate=True)
    rowptr, col = plan.csr()
    rng = np.random.default_rng(3)
    pts = rng.choice(plan.n_points, 20, replace=False)
    rows = point_rows(prob, pts)
    rp = rowptr.cpu().numpy()
    got, ref = [], []
    for g, (hs, blocks) in rows.items():
        for a in range(3):
            r0, r1 = rp[3 * g + a], rp[3 * g + a + 1]
            assert np.array_equal(col[r0:r1].cpu().numpy(), (3 * hs[:, None] + np.arange(3)).ravel())
            got.append(vals[r0:r1].double().cpu().numpy())
            ref.append(blocks[:, a, :].ravel())
    err = rel_fro(np.concatenate(got), np.concatenate(ref))
    print(prec, "beam4000 sampled", err)
    assert err <= TOL[prec], err


# ---------------------------------------------------------------- FP64 emulated on BF16 tensor cores
@pytest.mark.parametrize("n_e,q,n_tiles", [(2, 1, 1), (3, 3, 61), (2, 2, 8), (3, 0, 5)])
def test_f64_emu_contract_parity(n_e, q, n_tiles):
    """7 exact BF16 slices per operand: the FP64 bar (1e-12) on random data, where FP32-class
    arithmetic would give ~1e-7."""
    tab = msasm.Tables(synth.micro_cross(n_e), q)
    coef = np.random.default_rng(4).normal(size=(9 * n_tiles, 9 * tab.n_pi))
    coef[:, ::7] *= 1e-3                            # a spread of magnitudes within rows
    nz = blocks_to_rows(tab.contract(torch.tensor(coef, device="cuda"), "f64_emu").cpu().numpy())
    ref = coef @ oracle_table(n_e, q).reshape(tab.n_nz, -1).T
    err = rel_fro(nz, ref)
    print("f64_emu", n_e, q, n_tiles, err)
    assert err <= 1e-12, err


@pytest.mark.parametrize("name", ["cube8", "beam3x2x2_q3", "ragged_5x1x3_ne3_q2"])
def test_f64_emu_assemble_parity(name):
    from test_gpu_parity import make_case
    prob, tab, plan, ctrl = make_case(name)
    vals = plan.assemble(ctrl, 1.0, 0.3, "f64_emu", check_degenerate=True).cpu().numpy()
    err = rel_fro(vals, prob.assemble_lookup())
    print("f64_emu assemble", name, err)
    assert err <= 1e-12, err


def test_f64_emu_beam1000_full_size_sampled():
    w = synth.workload("beam1000")
    micro = synth.micro_cross(3)
    prob = Problem(micro, w.macro, 3, table=oracle_table(3, 3), structure=False)
    tab = msasm.Tables(micro, 3)
    plan = msasm.Plan(tab, w.macro)
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    vals = plan.assemble(ctrl, 1.0, 0.3, "f64_emu", check_degenerate=True)
    ref64 = plan.assemble(ctrl, 1.0, 0.3, "f64")
    full = (torch.linalg.vector_norm(vals - ref64) / torch.linalg.vector_norm(ref64)).item()
    rowptr, col = plan.csr()
    pts = np.random.default_rng(9).choice(plan.n_points, 24, replace=False)
    rows = point_rows(prob, pts)
    rp = rowptr.cpu().numpy()
    got, ref = [], []
    for g, (hs, blocks) in rows.items():
        for a in range(3):
            r0, r1 = rp[3 * g + a], rp[3 * g + a + 1]
            got.append(vals[r0:r1].cpu().numpy())
            ref.append(blocks[:, a, :].ravel())
    err = rel_fro(np.concatenate(got), np.concatenate(ref))
    print("f64_emu beam1000 sampled vs oracle", err, "whole matrix vs DFMA form", full)
    assert err <= 1e-12 and full <= 1e-12
