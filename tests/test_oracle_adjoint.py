"""Pins of the oracle's sensitivity u^T (dK/dP) u (Sec. 4.1.2) by properties of the exact map."""
import numpy as np
import pytest

import synth
from oracle import adjoint, tables
from oracle.assembly import Problem
from oracle.micro import ReferenceTile

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def prob():
    micro = synth.micro_cross(2)
    T = tables.build_table(ReferenceTile(micro), 1)
    return Problem(micro, synth.macro_twisted_beam(2, 1, 1), 1, table=T, structure=False)


def test_quadratic_form_matches_assembled_matrix():
    micro = synth.micro_cross(2)
    P = Problem(micro, synth.macro_perturbed_cube(seed=0), 1)
    u = np.random.default_rng(0).normal(size=(P.n_points, 3))
    v = P.assemble_lookup()
    row = np.repeat(np.arange(len(P.rowptr) - 1), np.diff(P.rowptr))
    q_csr = np.sum(v * u.ravel()[row] * u.ravel()[P.col])
    assert abs(adjoint.quadratic_form(P, u) - q_csr) < 1e-12 * abs(q_csr)


def test_complex_step_matches_central_differences(prob):
    u = np.random.default_rng(1).normal(size=(prob.n_points, 3))
    coords = [(3, 0), (17, 1), (40, 2), (63, 0), (25, 2)]
    cs = adjoint.gradient_complex_step(prob, u, coords)
    fd = adjoint.gradient_central_fd(prob, u, coords, h=1e-5)
    np.testing.assert_allclose(cs, fd, rtol=1e-6, atol=1e-8 * np.abs(cs).max())


def test_relative_form_equals_plain_form_and_removes_rigid_motion(prob):
    """The shifted per-tile form v^T K v (v = u - u[local point 0]) is the same function of P: on a
    random u both complex steps agree to rounding, and adding a large translation to u changes the
    shifted form's result by rounding only (K annihilates translations)."""
    u = np.random.default_rng(4).normal(size=(prob.n_points, 3))
    coords = [(3, 0), (17, 1), (40, 2), (63, 0)]
    a = adjoint.gradient_complex_step(prob, u, coords)
    b = adjoint.gradient_complex_step(prob, u, coords, relative=True)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())
    c = adjoint.gradient_complex_step(prob, u + np.array([1e4, -3e4, 2e4]), coords, relative=True)
    np.testing.assert_allclose(c, b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_gradient_homogeneity_and_translation(prob):
    """K(L P) = L K(P) exactly (J -> L J, |det J| -> L^3, G -> G/L), so by Euler's theorem
    sum_a P_a . dQ/dP_a = Q; and translating the net leaves K unchanged, so sum_a dQ/dP_a = 0."""
    u = np.random.default_rng(2).normal(size=(prob.n_points, 3))
    g = adjoint.gradient_all(prob, u)
    Q = adjoint.quadratic_form(prob, u)
    P = prob.mmap.macro.ctrl
    assert abs(np.sum(P * g) - Q) < 1e-11 * abs(Q)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-11 * np.abs(g).max())


def test_traction_load_total_force_and_area():
    """sum_A R_A = 1 on the face, so the load sums to t x (area of the strut ends on the face):
    per tile (c1 - c0)^2 times the area scaling of the (affine, sheared) macro map."""
    from oracle import loads
    m = synth.macro_affine_box(3, 2, 2)
    F = np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]])
    m.ctrl = m.ctrl @ F.T
    P = Problem(synth.micro_cross(2), m, 1, structure=False)
    t = np.array([0.3, -1.0, 0.5])
    f = loads.traction_load(P, 1, t)                       # face xi_1 = 1
    # area of a unit square in the (xi_2, xi_3) plane mapped by F
    area_unit = np.linalg.norm(np.cross(F[:, 1], F[:, 2]))
    expect = t * 4 * (0.3 ** 2) * area_unit               # 2 x 2 tiles on the face
    np.testing.assert_allclose(f.sum(axis=0), expect, rtol=1e-13, atol=1e-14)
    pts = loads.face_points(P, 1)
    assert len(pts) == 4 * 16 and np.all(np.abs(f[np.setdiff1d(np.arange(P.n_points), pts)]) == 0)


def test_mlp_oracle_gradient_fd_and_closed_form():
    from oracle import mlp
    H, n_out, B = 6, 5, 4
    rng = np.random.default_rng(7)
    p = rng.normal(size=mlp.n_params(H, n_out)) * 0.5
    x = rng.normal(size=B)
    t = rng.normal(size=(B, n_out))
    L, g = mlp.loss_grad(p, H, n_out, x, t)
    h = 1e-6
    for i in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p); e[i] = h
        fd = (mlp.loss_grad(p + e, H, n_out, x, t)[0] - mlp.loss_grad(p - e, H, n_out, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-8 * max(1.0, abs(g[i]))
    # zero output weights: y = b3, so dL/db3 = 2 sum_b (b3 - t_b) / (B n_out) and dL/dW1 = 0
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, H, n_out)
    W3[:] = 0.0
    L0, g0 = mlp.loss_grad(p, H, n_out, x, t)
    np.testing.assert_allclose(g0[-n_out:], 2 * (B * b3 - t.sum(0)) / (B * n_out), rtol=1e-13)
    assert np.all(g0[:H] == 0.0)
