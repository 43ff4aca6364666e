"""Pins of the oracle's traction load through the face lookup table (eq. 53-55 with F >= 1,
eq. 87-88): against the direct quadrature of the traction on the micro patch faces."""
import numpy as np
import pytest

import synth
from oracle import loads, quadrature, tables
from oracle.assembly import Problem

pytestmark = pytest.mark.filterwarnings("ignore")


def _affine():
    m = synth.macro_affine_box(2, 1, 1)
    m.ctrl = m.ctrl @ np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]]).T
    return m


def test_face_table_rows_and_closed_form_sums():
    """Only the points on the face have nonzero rows, and sum_A F[A, C2] is the integral of N_C2
    over the strut end face [0.5 - w/2, 0.5 + w/2]^2 (the basis sums to one): the product of two
    1-D integrals of Lagrange polynomials, integrated exactly here by their antiderivatives."""
    w = 0.3
    tile = Problem(synth.micro_cross(2, w), _affine(), 1, structure=False).tile
    q = 2
    g = quadrature.interp_nodes(q)
    lo, hi = 0.5 - w / 2, 0.5 + w / 2
    one_d = []
    for c in range(q + 1):
        others = [g[k] for k in range(q + 1) if k != c]
        poly = np.polynomial.Polynomial.fromroots(others) / np.prod([g[c] - x for x in others])
        P = poly.integ()
        one_d.append(P(hi) - P(lo))
    ref = np.array([one_d[ca] * one_d[cb] for cb in range(q + 1) for ca in range(q + 1)])
    for face in range(6):
        F = tables.face_load_table(tile, q, face)
        rows = np.nonzero(np.abs(F).sum(axis=1))[0]
        assert sorted(rows) == sorted(tile.faces[face])
        assert np.abs(F.sum(axis=0) - ref).max() <= 1e-15
        assert abs(F.sum() - w * w) <= 1e-15


@pytest.mark.parametrize("q", [0, 2])
@pytest.mark.parametrize("face", [1, 2, 5])
def test_affine_map_lookup_equals_direct_quadrature(q, face):
    """An affine macro map has a constant area element on every face: the projected traction is
    exact and the lookup form equals the quadrature of the traction on the patch faces."""
    prob = Problem(synth.micro_cross(2), _affine(), 1, structure=False)
    tr = (0.3, -1.0, 0.5)
    direct = loads.traction_load(prob, face, tr)
    look = loads.traction_load_lookup(prob, face, tr, q)
    assert np.abs(look - direct).max() <= 1e-14 * np.abs(direct).max()


def test_curved_face_converges_with_the_degree():
    """On a twisted face the area element varies; the lookup form converges to the quadrature."""
    prob = Problem(synth.micro_cross(2), synth.macro_twisted_beam(3, 2, 2), 1, structure=False)
    tr = (0.0, 0.0, -1.0)
    direct = loads.traction_load(prob, 3, tr)
    err = {q: np.abs(loads.traction_load_lookup(prob, 3, tr, q) - direct).max() / np.abs(direct).max()
           for q in (2, 4)}
    assert err[4] < 1e-5 and err[4] < 0.1 * err[2]
    total = loads.traction_load_lookup(prob, 3, tr, 4).sum(axis=0)
    assert abs(total[2] - direct.sum(axis=0)[2]) <= 1e-5 * abs(direct.sum())
