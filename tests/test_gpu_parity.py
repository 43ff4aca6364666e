"""GPU parity of every step of the hot path against the FP64 oracle (through the C ABI).

Tolerances: integer work (numbering, CSR pattern) bit-exact; FP64 forms relative
Frobenius <= 1e-12 (the kernels' own arithmetic is FP64 end to end, so the
measured gap is rounding order only, ~1e-15); FP32 CUDA-core form <= 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import tables as otables
from oracle import pullback as opullback
from oracle.assembly import Problem, point_rows, coefficient_block, nzdata_lookup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402

TOL = {"f64": 1e-12, "f64_emu": 1e-12, "f32": 1e-6}
_TABLE_CACHE = {}


def oracle_table(n_e, q, width=0.3):
    key = (n_e, q, width)
    if key not in _TABLE_CACHE:
        from oracle.micro import ReferenceTile
        _TABLE_CACHE[key] = otables.build_table(ReferenceTile(synth.micro_cross(n_e, width)), q)
    return _TABLE_CACHE[key]



def blocks_to_rows(nz):
    """The library's tile blocks (n_tiles, n_nz, 3, 3) as the rows nz[9t + 3a + b][m] of coef @ T^T."""
    t, m = nz.shape[:2]
    return nz.reshape(t, m, 9).transpose(0, 2, 1).reshape(9 * t, m)

def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def sheared_box(nx, ny, nz):
    m = synth.macro_affine_box(nx, ny, nz)
    F = np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]])
    m.ctrl = m.ctrl @ F.T
    return m


CASES = {
    "cube8": lambda: (2, 2, synth.macro_perturbed_cube(seed=0)),
    "beam3x2x2_q3": lambda: (2, 3, synth.macro_twisted_beam(3, 2, 2)),
    "single_tile_q1": lambda: (2, 1, synth.macro_twisted_beam(1, 1, 1)),
    "ragged_5x1x3_ne3_q2": lambda: (3, 2, synth.macro_twisted_beam(5, 1, 3)),
    "affine_q0": lambda: (2, 0, sheared_box(2, 2, 1)),
}


@pytest.fixture(scope="module")
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    msasm.load()
    return True


def make_case(name, tiles_per_pass=0):
    n_e, q, macro = CASES[name]()
    micro = synth.micro_cross(n_e)
    prob = Problem(micro, macro, q, table=oracle_table(n_e, q))
    tab = msasm.Tables(micro, q)
    plan = msasm.Plan(tab, macro, max_tiles_per_pass=tiles_per_pass)
    ctrl = torch.tensor(macro.ctrl, dtype=torch.float64, device="cuda")
    return prob, tab, plan, ctrl


# ---------------------------------------------------------------- step 2: table (K1)
@pytest.mark.parametrize("n_e,q", [(2, 2), (3, 3), (2, 3), (3, 0), (2, 1), (2, 5)])
def test_table_parity(built, n_e, q):
    tab = msasm.Tables(synth.micro_cross(n_e), q)
    T = tab.table().cpu().numpy()
    ref = oracle_table(n_e, q)
    assert T.shape == ref.shape
    assert np.abs(T - ref).max() <= 1e-13 * np.abs(ref).max()
    from oracle.micro import ReferenceTile
    assert np.array_equal(tab.pairs(), ReferenceTile(synth.micro_cross(n_e)).pairs)


def test_table_graded_width(built):
    for w in (0.15, 0.4):
        tab = msasm.Tables(synth.micro_cross(3, w), 3)
        ref = oracle_table(3, 3, w)
        assert np.abs(tab.table().cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------- integer structure (K6): bit-exact
@pytest.mark.parametrize("name", list(CASES))
def test_numbering_and_csr_bit_exact(built, name):
    prob, tab, plan, _ = make_case(name)
    assert plan.n_points == prob.n_points and plan.nnz == prob.nnz
    assert np.array_equal(plan.numbering().cpu().numpy(), prob.gmap.astype(np.int32))
    rowptr, col = plan.csr()
    assert np.array_equal(rowptr.cpu().numpy(), prob.rowptr)
    assert np.array_equal(col.cpu().numpy(), prob.col)


# ---------------------------------------------------------------- step 1: pullback (K2)
@pytest.mark.parametrize("name", ["cube8", "beam3x2x2_q3", "ragged_5x1x3_ne3_q2"])
def test_pullback_parity(built, name):
    prob, tab, plan, ctrl = make_case(name)
    coef = plan.pullback(ctrl, 1.0, 0.3).cpu().numpy()
    for t in range(plan.n_tiles):
        ref = coefficient_block(prob.mmap, t, prob.q, prob.lam, prob.mu).T     # (9, 9 n_pi)
        got = coef[9 * t:9 * t + 9]
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), t
    # eq. 38: A_ij = A_ji^T at every node
    n_pi = tab.n_pi
    A = coef.reshape(plan.n_tiles, 3, 3, n_pi, 3, 3)          # [t, a, b, C, i, j]
    assert np.abs(A - A.transpose(0, 2, 1, 3, 5, 4)).max() <= 1e-14 * np.abs(A).max()


def test_pullback_cube_closed_form(built):
    """eq. 98-100 through the GPU kernel: M = L xi gives the constant field of eq. 99."""
    L = 2.0
    m = synth.macro_affine_box(1, 1, 1, size=(L, L, L))
    tab = msasm.Tables(synth.micro_cross(2), 2)
    plan = msasm.Plan(tab, m)
    coef = plan.pullback(torch.tensor(m.ctrl, device="cuda"), 1.0, 0.3).cpu().numpy()
    lam, mu = opullback.lame(1.0, 0.3)
    A = coef.reshape(3, 3, tab.n_pi, 3, 3)                    # [a, b, C, i, j]
    a1, a2, a3 = (lam + 2 * mu) * L, mu * L, lam * L
    for C_ in range(tab.n_pi):
        np.testing.assert_allclose(A[:, :, C_, 0, 0], np.diag([a1, a2, a2]), atol=1e-14)
        np.testing.assert_allclose(A[:, :, C_, 1, 1], np.diag([a2, a1, a2]), atol=1e-14)
        np.testing.assert_allclose(A[:, :, C_, 0, 1], [[0, a3, 0], [a2, 0, 0], [0, 0, 0]], atol=1e-14)


# ---------------------------------------------------------------- step 3: contraction (K3)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n_e,q,n_tiles", [(2, 2, 8), (3, 3, 23), (2, 1, 1)])
def test_contract_parity(built, prec, n_e, q, n_tiles):
    tab = msasm.Tables(synth.micro_cross(n_e), q)
    rng = np.random.default_rng(7)
    coef = rng.normal(size=(9 * n_tiles, 9 * tab.n_pi))
    nz = blocks_to_rows(tab.contract(torch.tensor(coef, device="cuda"), prec).cpu().numpy())
    ref = coef @ oracle_table(n_e, q).reshape(tab.n_nz, -1).T
    assert rel_fro(nz, ref) <= TOL[prec]


# ---------------------------------------------------------------- full path (K2 -> K3 -> K5)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_assemble_parity(built, name, prec):
    prob, tab, plan, ctrl = make_case(name)
    vals = plan.assemble(ctrl, 1.0, 0.3, prec, check_degenerate=True).cpu().numpy()
    ref = prob.assemble_lookup()
    assert rel_fro(vals, ref) <= TOL[prec]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f64_emu", 1e-12), ("split_f16", 2e-6)])
@pytest.mark.parametrize("per_pass", [1, 3, 5])
def test_assemble_in_passes(built, per_pass, prec, tol):
    """Tile chunking (scratch for fewer tiles than the mesh; the glued-face contributions of a later
    pass are added to rows an earlier pass wrote) gives the same values."""
    prob, tab, plan, ctrl = make_case("beam3x2x2_q3", tiles_per_pass=per_pass)
    vals = plan.assemble(ctrl, 1.0, 0.3, prec).cpu().numpy()
    assert rel_fro(vals, prob.assemble_lookup()) <= tol


def test_scatter_stage(built):
    """Step 4 alone from the oracle's own nzdata."""
    prob, tab, plan, ctrl = make_case("cube8")
    nz = nzdata_lookup(prob.T, prob.mmap, prob.q, prob.lam, prob.mu)      # (t, m, a, b): the library's layout
    vals = plan.scatter(torch.tensor(np.ascontiguousarray(nz), device="cuda"), "f64").cpu().numpy()
    assert rel_fro(vals, prob.assemble_lookup()) <= 1e-14


@pytest.mark.parametrize("name,prec,per_pass", [("cube8", "f64", 0), ("beam3x2x2_q3", "f64_emu", 0),
                                                ("beam3x2x2_q3", "f64_emu", 1), ("ragged_5x1x3_ne3_q2", "f32", 0),
                                                ("ragged_5x1x3_ne3_q2", "split_f16", 2)])
def test_assemble_host_buffers(built, name, prec, per_pass):
    """Host-buffer entry point (passes with overlapped device-to-host copies of finished rows)
    returns exactly the device result, also with one or two tiles per pass."""
    prob, tab, plan, ctrl = make_case(name, tiles_per_pass=per_pass)
    dev = plan.assemble(ctrl, 1.0, 0.3, prec).cpu()
    h_ctrl = torch.tensor(prob.mmap.macro.ctrl).pin_memory()
    h_vals = torch.full((plan.nnz,), float("nan"), dtype=dev.dtype).pin_memory()
    plan.assemble_host(h_ctrl, h_vals, 1.0, 0.3, prec)
    assert torch.equal(dev, h_vals)


def test_translation_null_space_and_symmetry(built):
    prob, tab, plan, ctrl = make_case("beam3x2x2_q3")
    vals = plan.assemble(ctrl, 1.0, 0.3, "f64")
    rowptr, col = plan.csr()
    K = torch.sparse_csr_tensor(rowptr, col.long(), vals, size=(plan.n_rows, plan.n_rows))
    for a in range(3):
        u = torch.zeros(plan.n_points, 3, dtype=torch.float64, device="cuda")
        u[:, a] = 1.0
        r = K @ u.reshape(-1)
        assert r.abs().max().item() <= 1e-13 * vals.abs().max().item()
    Kd = K.to_dense()
    assert (Kd - Kd.T).abs().max().item() <= 1e-15 * 10 * vals.abs().max().item()


# ---------------------------------------------------------------- full-size launch (sampled outputs)
@pytest.mark.parametrize("prec", ["f64", "f64_emu", "f32"])
def test_beam1000_full_size_sampled(built, prec):
    """The 10x10x10 twisted beam, n_e = 3, q = 3, in the bench's launch configuration
    (all 1000 tiles in one pass, into a NaN-filled buffer): every value written, exact pattern
    and values of sampled rows."""
    w = synth.workload("beam1000")
    micro = synth.micro_cross(3)
    prob = Problem(micro, w.macro, 3, table=oracle_table(3, 3), structure=False)
    tab = msasm.Tables(micro, 3)
    plan = msasm.Plan(tab, w.macro)
    assert plan.nnz == 403850700 and plan.n_points == 657500
    ctrl = torch.tensor(w.macro.ctrl, device="cuda")
    out = torch.full((plan.nnz,), float("nan"), dtype=plan.value_dtype(prec), device="cuda")
    vals = plan.assemble(ctrl, 1.0, 0.3, prec, out=out, check_degenerate=True)
    assert not torch.isnan(vals).any().item()
    rowptr, col = plan.csr()
    rng = np.random.default_rng(11)
    pts = np.unique(np.concatenate([rng.choice(plan.n_points, 24, replace=False),
                                    prob.gmap[0, :3], prob.gmap[-1, -3:], prob.gmap[555, prob.tile.faces[0]][:4]]))
    rows = point_rows(prob, pts)
    rp = rowptr.cpu().numpy()
    got_all, ref_all = [], []
    for g, (hs, blocks) in rows.items():
        for a in range(3):
            r0, r1 = rp[3 * g + a], rp[3 * g + a + 1]
            c = col[r0:r1].cpu().numpy()
            assert np.array_equal(c, (3 * hs[:, None] + np.arange(3)[None, :]).ravel())
            got_all.append(vals[r0:r1].double().cpu().numpy())
            ref_all.append(blocks[:, a, :].ravel())
    assert rel_fro(np.concatenate(got_all), np.concatenate(ref_all)) <= TOL[prec]
    # translation null space on the whole matrix (a property that holds at any size)
    K = torch.sparse_csr_tensor(rowptr, col.long(), vals.double(), size=(plan.n_rows, plan.n_rows))
    u = torch.zeros(plan.n_points, 3, dtype=torch.float64, device="cuda")
    u[:, 1] = 1.0
    r = (K @ u.reshape(-1)).abs().max().item()
    assert r <= (1e-12 if prec in ("f64", "f64_emu") else 1e-5) * vals.abs().max().item()


# ---------------------------------------------------------------- failure paths
def test_degenerate_macro_element_is_reported(built):
    m = synth.macro_affine_box(2, 1, 1)
    m.ctrl = m.ctrl.copy()
    m.ctrl[:, 2] = 0.0                     # flatten the map: det J = 0 everywhere
    tab = msasm.Tables(synth.micro_cross(2), 1)
    plan = msasm.Plan(tab, m)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    with pytest.raises(msasm.MsasmError) as e:
        plan.assemble(ctrl, check_degenerate=True)
    assert e.value.status == -4
    plan.assemble(torch.tensor(synth.macro_affine_box(2, 1, 1).ctrl, device="cuda"), check_degenerate=True)
    assert plan.degenerate_count() == 0


def test_invalid_arguments(built):
    prob, tab, plan, ctrl = make_case("single_tile_q1")
    with pytest.raises(msasm.MsasmError) as e:
        plan.assemble(ctrl, E=-1.0)
    assert e.value.status == -1
    with pytest.raises(msasm.MsasmError):
        plan.assemble(ctrl, nu=0.5)
    with pytest.raises(msasm.MsasmError):
        msasm.Tables(synth.micro_cross(2), 7)
    # a values buffer that starts one value into an allocation (8-byte, not 16-byte aligned)
    buf = torch.empty(plan.nnz + 1, dtype=torch.float64, device="cuda")
    assert torch.equal(plan.assemble(ctrl, out=buf[1:]), plan.assemble(ctrl))
