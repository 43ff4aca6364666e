"""Pins of the oracle's projection error (eq. 59) and degree choice (eq. 65)."""
import numpy as np
import pytest

import synth
from oracle import projection, pullback, quadrature
from oracle.macro import MacroMap

pytestmark = pytest.mark.filterwarnings("ignore")


def test_affine_map_is_projected_exactly():
    """An affine macro map has a constant macro field, which every interpolation degree reproduces."""
    m = synth.macro_affine_box(2, 1, 1)
    m.ctrl = m.ctrl @ np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]]).T
    for q in (0, 1, 3):
        assert projection.projection_error(m, q)[1] < 1e-14


def test_interpolant_reproduces_the_nodes():
    """At the interpolation nodes themselves the error is zero (Kronecker property of the basis)."""
    m = synth.macro_perturbed_cube(seed=0)
    lam, mu = pullback.lame(1.0, 0.3)
    mm = MacroMap(m)
    for q in (1, 3):
        e = projection.tile_projection_error(mm, 0, q, lam, mu, points=quadrature.tensor_nodes(q))
        assert e < 1e-14


def test_error_decreases_with_degree_and_selection():
    m = synth.macro_twisted_beam(4, 2, 2)
    errs = [projection.projection_error(m, q)[1] for q in range(0, 6)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    tol = 0.5 * (errs[2] + errs[3])
    assert projection.select_degree(m, tol, 0, 5) == 3


def test_invariant_under_rotation_and_scaling_of_the_net():
    """Rotating the net rotates the macro field's alpha, beta indices (an orthogonal change of basis that
    keeps the Frobenius norms); scaling it by L scales the field by L: the relative error is unchanged."""
    m = synth.macro_perturbed_cube(seed=2)
    e0 = projection.projection_error(m, 2)[0]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    np.testing.assert_allclose(projection.projection_error(m, 2, ctrl=3.0 * m.ctrl @ R.T)[0], e0, rtol=1e-10)


# ---------------------------------------------------------------- L2 projection (eq. 20-24)
def _tile_field(mm, t, xi, lam, mu):
    _, J = mm.tile_map(t, xi)
    return pullback.macro_field(J, lam, mu).reshape(len(xi), 81)


def test_l2_with_the_nodes_own_rule_is_interpolation():
    """With the (q+1)-point Gauss rule for the load, the L2 projection is the interpolant at the
    nodes: the rule's points are the nodes and the mass matrix is diagonal with its weights."""
    m = synth.macro_twisted_beam(3, 2, 2)
    lam, mu = pullback.lame(1.0, 0.3)
    mm = MacroMap(m)
    for q in (0, 1, 3):
        a = projection.l2_coefficients(mm, 4, q, lam, mu, q + 1)
        nodes = _tile_field(mm, 4, quadrature.tensor_nodes(q), lam, mu)
        assert np.abs(a - nodes).max() <= 1e-13 * np.abs(nodes).max()


def test_l2_reproduces_a_constant_field():
    """An affine macro map has a constant field, which the projection onto Q_q returns exactly."""
    m = synth.macro_affine_box(2, 1, 1)
    m.ctrl = m.ctrl @ np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]]).T
    lam, mu = pullback.lame(1.0, 0.3)
    mm = MacroMap(m)
    const = _tile_field(mm, 1, np.array([[0.3, 0.6, 0.2]]), lam, mu)[0]
    for q, n_g in ((0, 3), (2, 5), (3, 6)):
        a = projection.l2_coefficients(mm, 1, q, lam, mu, n_g)
        assert np.abs(a - const[None, :]).max() <= 1e-13 * np.abs(const).max()


def test_l2_is_the_best_approximation_in_its_norm():
    """On a curved tile the L2 coefficients (load by the n-point rule) minimise the n-point discrete
    L2 norm of the error over Q_q: every perturbation of them raises it, and the interpolant's
    error is larger."""
    m = synth.macro_twisted_beam(3, 2, 2)
    lam, mu = pullback.lame(1.0, 0.3)
    mm = MacroMap(m)
    q, n = 2, 7
    xg, wg = projection.tensor_gauss(n)
    F = _tile_field(mm, 5, xg, lam, mu)
    N = quadrature.tensor_lagrange(q, xg)
    err = lambda a: float(np.sum(wg[:, None] * (F - N @ a) ** 2))
    a = projection.l2_coefficients(mm, 5, q, lam, mu, n)
    e0 = err(a)
    rng = np.random.default_rng(3)
    for _ in range(8):
        d = rng.standard_normal(a.shape) * 1e-6 * np.abs(a).max()
        assert err(a + d) > e0
    nodes = _tile_field(mm, 5, quadrature.tensor_nodes(q), lam, mu)
    assert err(nodes) > e0 * (1 + 1e-6)


def test_l2_converges_in_the_load_rule_and_beats_interpolation_on_samples():
    """The coefficients converge as the load rule grows (smooth field); on this beam the sampled
    error of eq. 59 is also below the interpolant's (an observation, not a theorem: the projection
    minimises the L2 norm, not the largest sampled error)."""
    m = synth.macro_twisted_beam(3, 2, 2)
    lam, mu = pullback.lame(1.0, 0.3)
    mm = MacroMap(m)
    a8 = projection.l2_coefficients(mm, 7, 3, lam, mu, 8)
    a10 = projection.l2_coefficients(mm, 7, 3, lam, mu, 10)
    assert np.abs(a8 - a10).max() <= 1e-9 * np.abs(a10).max()
    e_int = projection.projection_error(m, 1)[1]
    e_l2 = projection.projection_error(m, 1, n_gauss=6)[1]
    assert 0 < e_l2 < e_int
