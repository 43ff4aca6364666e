"""Pins of the oracle with a projection degree per direction (q1, q2, q3) (the anisotropic
projection space of Sec. 3.3.4; eq. 20-24, 42, 52, 59, 65 with Q_q replaced by Q_(q1,q2,q3))."""
import numpy as np
import pytest

import synth
from oracle import projection, quadrature, tables
from oracle.micro import ReferenceTile

pytestmark = pytest.mark.filterwarnings("ignore")


def test_tensor_interpolation_is_exact_exactly_up_to_the_degrees():
    """The interpolant in Q_(1,3,2) reproduces xi1^a xi2^b xi3^c iff a <= 1, b <= 3, c <= 2."""
    q = (1, 3, 2)
    nodes = quadrature.tensor_nodes(q)
    assert nodes.shape == (2 * 4 * 3, 3)
    x = np.random.default_rng(0).uniform(size=(50, 3))
    N = quadrature.tensor_lagrange(q, x)
    for a, b, c in [(1, 3, 2), (0, 2, 1), (2, 0, 0), (0, 4, 0), (0, 0, 3)]:
        f = lambda p: p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c
        err = np.abs(N @ f(nodes) - f(x)).max()
        if a <= 1 and b <= 3 and c <= 2:
            assert err <= 1e-13
        else:
            assert err > 1e-4


def _ordered_sum(tile, T):
    full = np.zeros((tile.n_T,) + T.shape[1:])
    for m, (A, B) in enumerate(tile.pairs):
        full[A] += T[m]
        if A != B:
            full[B] += T[m].transpose(0, 2, 1)
    return full


def test_anisotropic_tables():
    """Equal degrees give the isotropic tables exactly; Q_(1,3,2): partition of unity of the
    stiffness table (sum over B vanishes), the volume table sums to the tile volume
    w^3 + 3 w^2 (1 - w), and the load table rows sum to the volume table."""
    tile = ReferenceTile(synth.micro_cross(2))
    assert np.array_equal(tables.build_table(tile, (2, 2, 2)), tables.build_table(tile, 2))
    q = (1, 3, 2)
    T = tables.build_table(tile, q)
    assert T.shape[1] == 24
    assert np.abs(_ordered_sum(tile, T)).max() <= 1e-12 * np.abs(T).max()
    vol = tables.volume_table(tile, q)
    w = 0.3
    assert abs(vol.sum() - (w ** 3 + 3 * w ** 2 * (1 - w))) <= 1e-15
    assert np.abs(tables.load_table(tile, q).sum(axis=0) - vol).max() <= 1e-15
    for face in (0, 3, 4):
        F = tables.face_load_table(tile, q, face)
        d = face // 2
        qa, qb = [q[k] for k in range(3) if k != d]
        assert F.shape == (tile.n_T, (qa + 1) * (qb + 1)) and abs(F.sum() - w * w) <= 1e-15


def test_anisotropic_projection_error():
    beam = synth.macro_twisted_beam(3, 2, 2)
    e_iso = projection.projection_error(beam, 2)[1]
    assert projection.projection_error(beam, (2, 2, 2))[1] == e_iso
    affine = synth.macro_affine_box(2, 1, 1)
    affine.ctrl = affine.ctrl @ np.array([[1.0, 0.2, 0.1], [0.0, 0.8, 0.3], [0.1, 0.0, 1.3]]).T
    assert projection.projection_error(affine, (0, 1, 2))[1] < 1e-14


def test_degree_selection_per_direction():
    """The selected degrees meet the tolerance and none of them can be lowered alone."""
    beam = synth.macro_twisted_beam(4, 2, 2)
    tol = 1e-3
    q, err = projection.select_degrees(beam, tol, (3, 3, 3))
    assert projection.meets(err, tol) and projection.projection_error(beam, q)[1] == err
    for d in range(3):
        if q[d] > 0:
            c = list(q)
            c[d] -= 1
            assert not projection.meets(projection.projection_error(beam, tuple(c))[1], tol)
