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
