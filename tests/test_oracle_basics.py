"""Pins of the oracle's building blocks against closed forms and independent libraries."""
import numpy as np
import pytest
import scipy.interpolate

import synth
from oracle import bspline, quadrature, pullback
from oracle.micro import ReferenceTile

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- B-splines (eq. 1-4)
@pytest.mark.parametrize("p,knots", [
    (2, [0, 0, 0, 0.5, 1, 1, 1]),
    (3, [0, 0, 0, 0, 0.25, 0.5, 0.75, 1, 1, 1, 1]),
    (3, [0, 0, 0, 0, 0.3, 0.3, 0.8, 1, 1, 1, 1]),
    (2, [0, 0, 0, 1 / 3, 2 / 3, 1, 1, 1]),
])
def test_bspline_matches_scipy_and_partition_of_unity(p, knots):
    knots = np.array(knots, float)
    u = np.linspace(0, 1, 41)
    N = bspline.basis(knots, p, u)
    D = bspline.basis_deriv(knots, p, u)
    n = len(knots) - p - 1
    for i in range(n):
        c = np.zeros(n); c[i] = 1.0
        s = scipy.interpolate.BSpline(knots, c, p, extrapolate=False)
        ref = np.nan_to_num(s(u))
        ref[-1] = s(1.0 - 1e-15)  # scipy leaves the closed right end undefined
        np.testing.assert_allclose(N[:, i], ref, atol=1e-13)
        dref = np.nan_to_num(s.derivative()(np.clip(u, 0, 1 - 1e-15)))
        np.testing.assert_allclose(D[:, i], dref, atol=1e-9)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-12)


def test_knot_insertion_keeps_geometry():
    """The refined 2x2x2 cube is the same map as the raw Bezier cube (input check)."""
    ref = synth.bezier_cube_reference(seed=0)
    ref2 = synth.macro_perturbed_cube(seed=0)
    u = np.random.default_rng(1).uniform(0, 1, (50, 3))
    x1, J1 = bspline.volume_eval(ref.knots, ref.degree, ref.ctrl, u)
    x2, J2 = bspline.volume_eval(ref2.knots, ref2.degree, ref2.ctrl, u)
    np.testing.assert_allclose(x1, x2, atol=1e-14)
    np.testing.assert_allclose(J1, J2, atol=1e-13)


def test_volume_eval_derivative_vs_fd():
    m = synth.macro_twisted_beam(3, 2, 2)
    u = np.array([[0.31, 0.52, 0.77]])
    _, J = bspline.volume_eval(m.knots, m.degree, m.ctrl, u)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3); e[d] = h
        xp, _ = bspline.volume_eval(m.knots, m.degree, m.ctrl, u + e)
        xm, _ = bspline.volume_eval(m.knots, m.degree, m.ctrl, u - e)
        np.testing.assert_allclose(J[0, :, d], (xp - xm)[0] / (2 * h), rtol=1e-7, atol=1e-8)


# ---------------------------------------------------------------- quadrature / interpolation
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_gauss_exact_on_monomials(n):
    x, w = quadrature.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-15
    assert abs(w @ x ** (2 * n) - 1.0 / (2 * n + 1)) > 1e-8   # and not one degree more


@pytest.mark.parametrize("q", [0, 1, 2, 3, 4])
def test_lagrange_reproduces_q(q):
    g = quadrature.interp_nodes(q)
    np.testing.assert_allclose(quadrature.lagrange(g, g), np.eye(q + 1), atol=1e-14)
    x = np.linspace(0, 1, 17)
    for k in range(q + 1):
        np.testing.assert_allclose(quadrature.lagrange(g, x) @ g ** k, x ** k, atol=1e-13)
    xi = np.random.default_rng(0).uniform(0, 1, (20, 3))
    L = quadrature.tensor_lagrange(q, xi)
    nodes = quadrature.tensor_nodes(q)
    f = lambda p: (1 + p[:, 0] ** q) * (2 - p[:, 1]) ** min(q, 1) * (p[:, 2] + 0.5) ** q
    np.testing.assert_allclose(L @ f(nodes), f(xi), rtol=1e-12)


# ---------------------------------------------------------------- reference tile (eq. 3, 56)
@pytest.mark.parametrize("n_e", [2, 3])
def test_reference_tile_counts(n_e):
    """Counts from first principles: 7 patches of (n_e+2)^3 points glued on 6 faces of
    (n_e+2)^2; 1-D degree-2 functions i, j share an element iff neither support ends before
    the other starts, giving s = (n_e+2)^2 - 2 * #{|i-j| >= 3 or disjoint} ordered 1-D pairs."""
    R = ReferenceTile(synth.micro_cross(n_e))
    n = n_e + 2
    s = sum(1 for i in range(n) for j in range(n)
            if max(i - 2, 0) <= min(j, n_e - 1) and max(j - 2, 0) <= min(i, n_e - 1))
    assert R.n_T == 7 * n ** 3 - 6 * n ** 2
    n_ordered = 7 * s ** 3 - 6 * s ** 2
    assert 2 * R.n_nz - R.n_T == n_ordered
    assert len(R.elements) == 7 * n_e ** 3
    assert {2: (352, 9192), 3: (725, 23286)}[n_e] == (R.n_T, R.n_nz)
    assert all(len(f) == n ** 2 for f in R.faces)
    # opposite faces match point for point
    for d in range(3):
        a, b = R.points[R.faces[2 * d]], R.points[R.faces[2 * d + 1]]
        od = [k for k in range(3) if k != d]
        np.testing.assert_allclose(a[:, od], b[:, od], atol=1e-12)


# ---------------------------------------------------------------- macro field (eq. 37, 99-100)
def _golden_eq99():
    rows = []
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cube_macro_field_eq99.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            i, j, a, b, c = line.split()
            rows.append((int(i) - 1, int(j) - 1, int(a) - 1, int(b) - 1, c))
    return rows


@pytest.mark.parametrize("L", [1.0, 2.5, 0.37])
def test_macro_field_cube_closed_form(L):
    """Appendix A.2.2: the affine cube has the constant field of eq. 99 with eq. 100."""
    lam, mu = pullback.lame(1.0, 0.3)
    A = pullback.macro_field(L * np.eye(3), lam, mu)
    coef = dict(a1=(lam + 2 * mu) * L, a2=mu * L, a3=lam * L)
    expect = np.zeros((3, 3, 3, 3))
    for i, j, a, b, c in _golden_eq99():
        expect[i, j, a, b] = coef[c]
        expect[j, i, b, a] = coef[c]          # eq. 38
    np.testing.assert_allclose(A, expect, atol=1e-14 * L)


def test_macro_field_symmetry_and_energy():
    """eq. 38 symmetry, and the quadratic form equals the isotropic energy density
    |det J| (lam tr(H) tr(K) + 2 mu sym(H):sym(K)) with H = u_,xi J^-1 (textbook elasticity)."""
    lam, mu = pullback.lame(2.0, 0.27)
    rng = np.random.default_rng(3)
    for _ in range(10):
        J = rng.normal(size=(3, 3)) + 2 * np.eye(3)
        A = pullback.macro_field(J, lam, mu)
        np.testing.assert_allclose(A, A.transpose(1, 0, 3, 2), atol=1e-12)
        du, dv = rng.normal(size=(3, 3)), rng.normal(size=(3, 3))   # [component, xi_i]
        quad = np.einsum("ai,ijab,bj->", du, A, dv)
        Hu, Hv = du @ np.linalg.inv(J), dv @ np.linalg.inv(J)
        su, sv = 0.5 * (Hu + Hu.T), 0.5 * (Hv + Hv.T)
        ref = abs(np.linalg.det(J)) * (lam * np.trace(Hu) * np.trace(Hv) + 2 * mu * np.sum(su * sv))
        assert abs(quad - ref) < 1e-11 * max(1.0, abs(ref))
        np.testing.assert_allclose(A, pullback.macro_field_cartesian(J, lam, mu), atol=1e-12)


def test_contravariant_material_symmetries():
    """eq. 84b: C^ijkl = C^jikl = C^ijlk = C^klij."""
    g = np.random.default_rng(5).normal(size=(3, 3))
    gcon = np.linalg.inv(g.T @ g)
    C = pullback.material_contravariant(gcon, 0.7, 0.4)
    np.testing.assert_allclose(C, C.transpose(1, 0, 2, 3), atol=1e-14)
    np.testing.assert_allclose(C, C.transpose(0, 1, 3, 2), atol=1e-14)
    np.testing.assert_allclose(C, C.transpose(2, 3, 0, 1), atol=1e-14)
