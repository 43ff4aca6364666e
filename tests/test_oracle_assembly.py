"""Pins of the oracle's table, numbering and both assembly forms (Sec. 3.2-3.3)."""
import numpy as np
import pytest

import synth
from oracle import tables, quadrature, pullback
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def tile2():
    return ReferenceTile(synth.micro_cross(2))


@pytest.fixture(scope="module")
def table2(tile2):
    return tables.build_table(tile2, 2)


def _ordered_sum(tile, T):
    """sum over B of the ordered-pair table rows, per A."""
    full = np.zeros((tile.n_T,) + T.shape[1:])
    for m, (A, B) in enumerate(tile.pairs):
        full[A] += T[m]
        if A != B:
            full[B] += T[m].transpose(0, 2, 1)
    return full


def test_table_partition_of_unity(tile2, table2):
    """sum_B d_j phi_B = 0, so summing eq. 52 over B vanishes for every A, C, i, j."""
    assert np.abs(_ordered_sum(tile2, table2)).max() < 1e-15 * 1e3 * np.abs(table2).max()


def test_table_quadrature_is_exact(tile2, table2):
    """The default rule already integrates the polynomial integrand exactly."""
    T8 = tables.build_table(tile2, 2, n_g=5)
    assert np.abs(T8 - table2).max() < 1e-15 * 50


def test_table_polynomial_moment_brute_force(tile2, table2):
    """For a field f in Q_q, sum_C f(xi_C) T[m, C, i, j] = int d_i phi_A d_j phi_B f, the
    right side integrated by a high-order rule directly in xi (independent path)."""
    q = 2
    f = lambda x: (1 + 2 * x[:, 0] - x[:, 0] ** 2) * (0.5 + x[:, 1] ** 2) * (2 - x[:, 2])
    lhs = np.einsum("mcij,c->mij", table2, f(quadrature.tensor_nodes(q)))
    rng = np.random.default_rng(0)
    ms = rng.choice(tile2.n_nz, 40, replace=False)
    g1, w1 = quadrature.gauss_legendre(8)
    for m in ms:
        A, B = tile2.pairs[m]
        val = np.zeros((3, 3))
        for el in tile2.elements:
            if A not in el["ids"] or B not in el["ids"]:
                continue
            P = tile2.patches[el["patch"]]
            lo, hi = P["lo"], P["hi"]
            pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
            wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
            th = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
            w = np.array([a * b * c for c in wts[2] for b in wts[1] for a in wts[0]]) * np.prod(hi - lo)
            _, gr = tile2.patch_basis(el["patch"], th)
            nf = P["nfun"]
            def col(X):
                a1, a2, a3 = el["loc"][el["ids"].index(X)]
                return a1 + nf[0] * (a2 + nf[1] * a3)
            dA, dB = gr[:, col(A), :] / (hi - lo), gr[:, col(B), :] / (hi - lo)
            val += np.einsum("g,gi,gj,g->ij", w, dA, dB, f(lo + (hi - lo) * th))
        np.testing.assert_allclose(lhs[m], val, atol=1e-15 * 100)


def test_volume_table_matches_cell_volume(tile2):
    """sum_C t_C = vol(Omega_T) = w^3 + 6 w^2 (1 - w)/2 (eq. 18 with sum_C N_C = 1)."""
    for q in (0, 2, 3):
        t = tables.volume_table(tile2, q)
        assert abs(t.sum() - (0.3 ** 3 + 3 * 0.3 ** 2 * 0.7)) < 1e-15 * 10


def test_volume_fraction_at_degree_zero(tile2):
    """Sec. 4.1.1: with p_pi = 0 the adjoint field equals the volume fraction."""
    t = tables.volume_table(tile2, 0)
    assert t.shape == (1,) and abs(t[0] - 0.216) < 1e-15 * 10


# ---------------------------------------------------------------- assembly
def _affine_problem(q=1, nx=2, ny=1, nz=1):
    m = synth.macro_affine_box(nx, ny, nz)
    F = np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]])
    m.ctrl = m.ctrl @ F.T
    return Problem(synth.micro_cross(2), m, q), F


def test_affine_lookup_equals_quadrature():
    """Affine macro map: constant A_ij, so interpolation is exact and both forms agree."""
    P, _ = _affine_problem(q=1)
    a, b = P.assemble_lookup(), P.assemble_quadrature(n_g=3)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-14


def _dense(P, v):
    n = len(P.rowptr) - 1
    K = np.zeros((n, n))
    for r in range(n):
        K[r, P.col[P.rowptr[r]:P.rowptr[r + 1]]] = v[P.rowptr[r]:P.rowptr[r + 1]]
    return K


def test_affine_rigid_modes_and_constant_strain_energy():
    P, F = _affine_problem(q=1, nx=2, ny=2, nz=1)
    K = _dense(P, P.assemble_lookup())
    X = P.point_positions()
    scale = np.abs(K).max()
    for a in range(3):                           # translations
        u = np.zeros_like(X); u[:, a] = 1.0
        assert np.abs(K @ u.ravel()).max() < 1e-13 * scale
    for w in np.eye(3):                          # rotations u = w x X
        u = np.cross(w, X)
        assert np.abs(K @ u.ravel()).max() < 1e-12 * scale * np.abs(X).max()
    eps = np.array([[0.3, 0.1, -0.2], [0.1, -0.4, 0.05], [-0.2, 0.05, 0.25]])
    u = X @ eps.T
    energy = 0.5 * u.ravel() @ K @ u.ravel()
    V = P.mmap.n_tiles * abs(np.linalg.det(F)) * 0.216
    # the macro box has unit tiles before F; each tile volume is |det F| * vol(Omega_T)
    expect = 0.5 * V * (P.lam * np.trace(eps) ** 2 + 2 * P.mu * np.sum(eps * eps))
    assert abs(energy - expect) < 1e-12 * expect


def test_symmetry_translation_and_counts_curved():
    w = synth.workload("cube8")
    P = Problem(synth.micro_cross(2), w.macro, 2)
    v = P.assemble_lookup()
    assert P.nnz == 1277136 and P.n_points == 2624
    # nnz = 9 (m_M * ordered pairs - interfaces * face pairs), face pairs = 14^2 for n_e = 2
    assert P.nnz == 9 * (8 * 18032 - 12 * 196)
    K = _dense(P, v)
    assert np.abs(K - K.T).max() < 1e-15 * 10 * np.abs(K).max()
    for a in range(3):
        u = np.zeros((P.n_points, 3)); u[:, a] = 1.0
        assert np.abs(K @ u.ravel()).max() < 1e-14 * 10 * np.abs(K).max()
    # col sorted unique per row
    for r in range(0, len(P.rowptr) - 1, 97):
        c = P.col[P.rowptr[r]:P.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.slow
def test_emat_decreases_with_q():
    """Fig. 7 trend: the lookup form converges to the quadrature form as q grows."""
    w = synth.workload("cube8")
    P = Problem(synth.micro_cross(2), w.macro, 0)
    ref = P.assemble_quadrature(n_g=5)
    errs = []
    for q in range(0, 5):
        P.T, P.q = tables.build_table(P.tile, q), q
        v = P.assemble_lookup()
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4    # Table 1 magnitudes are 1e-5 .. 1e-4 at degree 4


@pytest.mark.parametrize("name,n_points", [("beam1000", 657500), ("beam4000", 2622500),
                                           ("arc2000", 1312500), ("cantilever2000", 617600)])
def test_global_point_counts(name, n_points):
    """n_points = m_M n_T - (#interior tile faces) (n_e+2)^2: each glued face merges its points."""
    from oracle.assembly import numbering
    from oracle.macro import MacroMap
    w = synth.workload(name)
    R = ReferenceTile(synth.micro_cross(w.n_e))
    mm = MacroMap(w.macro)
    gmap, n = numbering(R, mm)
    nx, ny, nz = mm.n_elem
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert n == n_points == mm.n_tiles * R.n_T - faces * (w.n_e + 2) ** 2
    # ids are assigned in (owner tile, local id) order
    owned_first = [gmap[t][gmap[t] >= (gmap[t - 1].max() + 1 if t else 0)] for t in range(3)]
    for o in owned_first:
        assert np.all(np.diff(o) == 1)
