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


def test_gradient_homogeneity_and_translation(prob):
    """K(L P) = L K(P) exactly (J -> L J, |det J| -> L^3, G -> G/L), so by Euler's theorem
    sum_a P_a . dQ/dP_a = Q; and translating the net leaves K unchanged, so sum_a dQ/dP_a = 0."""
    u = np.random.default_rng(2).normal(size=(prob.n_points, 3))
    g = adjoint.gradient_all(prob, u)
    Q = adjoint.quadratic_form(prob, u)
    P = prob.mmap.macro.ctrl
    assert abs(np.sum(P * g) - Q) < 1e-11 * abs(Q)
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-11 * np.abs(g).max())
