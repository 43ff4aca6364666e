"""Pins of the oracle's volume (Sec. 3.1, eq. 14-19), volume gradient (Sec. 4.1.1, eq. 66-67) and
body-force load vector (eq. 53-55) by closed forms and invariants of the exact maps."""
import numpy as np
import pytest

import synth
from oracle import tables, volume
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def tile2():
    return ReferenceTile(synth.micro_cross(2))


def test_load_table_degree_zero_is_the_bspline_integral(tile2):
    """q = 0 (N = 1): F[A] = int R_A = sum over the patches holding A of prod_d h_d (t_{i+p+1} - t_i)/(p+1),
    the textbook integral of a B-spline, independent of any quadrature."""
    F = tables.load_table(tile2, 0)[:, 0]
    ref = np.zeros(tile2.n_T)
    for P in tile2.patches:
        nf = P["nfun"]
        for loc, A in enumerate(P["ids"]):
            idx = (loc % nf[0], (loc // nf[0]) % nf[1], loc // (nf[0] * nf[1]))
            v = 1.0
            for d in range(3):
                k, p, i = P["knots"][d], P["degree"][d], idx[d]
                v *= (P["hi"][d] - P["lo"][d]) * (k[i + p + 1] - k[i]) / (p + 1)
            ref[A] += v
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-15)
    assert abs(F.sum() - 0.216) < 1e-14


@pytest.mark.parametrize("q", [1, 2, 3])
def test_load_table_partition_of_unity_and_exactness(tile2, q):
    F = tables.load_table(tile2, q)
    np.testing.assert_allclose(F.sum(axis=0), tables.volume_table(tile2, q), rtol=0, atol=1e-15)
    p_T = max(max(P["degree"]) for P in tile2.patches)
    F2 = tables.load_table(tile2, q, n_g=tables.default_gauss_points(p_T, q) + 2)
    np.testing.assert_allclose(F, F2, rtol=0, atol=1e-15)


def _affine(q=1, nx=2, ny=2, nz=1):
    m = synth.macro_affine_box(nx, ny, nz)
    Fm = np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]])
    m.ctrl = m.ctrl @ Fm.T
    return Problem(synth.micro_cross(2), m, q, structure=False), Fm


@pytest.mark.parametrize("q", [0, 2])
def test_volume_affine_map_is_exact(q):
    """An affine macro map has constant |det J| = |det F|: every tile holds |det F| vol(Omega_T)."""
    prob, Fm = _affine(q)
    vt, V = volume.volume_lookup(prob)
    np.testing.assert_allclose(vt, abs(np.linalg.det(Fm)) * 0.216, rtol=1e-14)
    assert abs(volume.volume_quadrature(prob) - V) < 1e-13 * V


def test_volume_lookup_converges_to_quadrature():
    """Curved (perturbed cubic) macro map: the lookup volume approaches the full-quadrature volume
    (eq. 14) as the interpolation degree grows (the Sec. 3.1.3 trend)."""
    m = synth.macro_perturbed_cube(seed=0)
    errs = []
    for q in range(0, 5):
        prob = Problem(synth.micro_cross(2), m, q, structure=False)
        if q == 0:
            V_ref = volume.volume_quadrature(prob)
        errs.append(abs(volume.volume_lookup(prob)[1] - V_ref) / V_ref)
    # two more nodes per direction always help (odd and even degrees interleave: 1.2e-4, 4.9e-4,
    # 3.0e-6, 1.1e-5, 3.6e-8 here)
    assert all(errs[q + 2] < 0.1 * errs[q] for q in range(3)), errs
    assert errs[-1] < 1e-6, errs


def test_volume_gradient_invariants_and_fd():
    """Translation leaves V unchanged (sum of the gradient over control points is zero); scaling the net
    by L scales V by L^3 (Euler: sum P . dV/dP = 3 V); complex step agrees with central differences."""
    m = synth.macro_twisted_beam(2, 1, 1)
    prob = Problem(synth.micro_cross(2), m, 2, structure=False)
    n = m.ctrl.shape[0]
    coords = [(k, p) for k in range(n) for p in range(3)]
    g = volume.volume_gradient_complex_step(prob, coords).reshape(n, 3)
    V = volume.volume_lookup(prob)[1]
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-13 * np.abs(g).max())
    assert abs(np.sum(m.ctrl * g) - 3 * V) < 1e-12 * V
    h = 1e-6
    for k, p in [(3, 0), (17, 1), (40, 2)]:
        c = m.ctrl.copy(); c[k, p] += h
        vp = volume.volume_lookup(prob, c)[1]
        c[k, p] -= 2 * h
        vm = volume.volume_lookup(prob, c)[1]
        assert abs((vp - vm) / (2 * h) - g[k, p]) < 1e-7 * np.abs(g).max()


def test_body_load_total_force_and_affine_quadrature():
    """The control points' loads sum to b V (the basis functions sum to one); on an affine map each
    equals b |det F| int R_A."""
    b = np.array([0.3, -1.0, 0.2])
    m = synth.macro_perturbed_cube(seed=1)
    prob = Problem(synth.micro_cross(2), m, 2, structure=False)
    f = volume.body_load(prob, b)
    np.testing.assert_allclose(f.sum(axis=0), b * volume.volume_lookup(prob)[1], rtol=1e-13)
    prob, Fm = _affine(1, 1, 1, 1)
    f = volume.body_load(prob, b)
    ref = abs(np.linalg.det(Fm)) * tables.load_table(prob.tile, 0)[:, 0][:, None] * b[None, :]
    np.testing.assert_allclose(f[prob.gmap[0]], ref, rtol=0, atol=1e-14)
