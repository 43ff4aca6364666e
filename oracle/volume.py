"""Volume, its gradient and the body-force load vector through lookup tables (test infrastructure).

* Volume (Sec. 3.1, eq. 14-19): the macro-Jacobian determinant is replaced by its interpolant at the
  (q+1)^3 nodes, d_C^(t) = |det J^(t)(xi_C)| (the same reading of the projection as for the stiffness),
  so V^(t) = t^h . d^(t) (eq. 17) with t^h the volume table (eq. 18), and V = sum_t V^(t) (eq. 19).
* Volume gradient (Sec. 4.1.1, eq. 66-67): dV/dm = sum_t sum_C t_C d|det J^(t)(xi_C)|/dm, taken here
  by complex step of V (Squire and Trapp 1998).
* Body-force load (eq. 39-40, 53-55 with F = 0): for a constant body force b,
  b_bar^(t) = b |det J^(t)| is interpolated at the nodes, so the tile load of control point A is
  f_A^(t) = b sum_C F[A, C] d_C^(t); the global vector sums the tiles sharing a point.
* The standard quadrature volume (eq. 14) is the reference the lookup form converges to.
"""
from __future__ import annotations

import numpy as np

from . import quadrature, tables
from .assembly import node_jacobians


def node_abs_det(mmap, t, q, ctrl=None):
    """|det J^(t)(xi_C)| at the nodes (complex-safe: det times the sign of its real part)."""
    J = node_jacobians(mmap, t, q, ctrl)
    det = np.linalg.det(J) if not np.iscomplexobj(J) else _det3(J)
    return det * np.sign(np.real(det))


def _det3(J):
    return (J[:, 0, 0] * (J[:, 1, 1] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 1])
            - J[:, 0, 1] * (J[:, 1, 0] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 0])
            + J[:, 0, 2] * (J[:, 1, 0] * J[:, 2, 1] - J[:, 1, 1] * J[:, 2, 0]))


def volume_lookup(prob, ctrl=None, t_h=None):
    """(per-tile volumes V^(t) (eq. 17), total V (eq. 19))."""
    t_h = tables.volume_table(prob.tile, prob.q) if t_h is None else t_h
    vt = np.array([t_h @ node_abs_det(prob.mmap, t, prob.q, ctrl) for t in range(prob.mmap.n_tiles)])
    return vt, vt.sum()


def volume_quadrature(prob, n_g=6, ctrl=None):
    """Eq. 14 by full Gauss quadrature over every micro element of every tile."""
    tile, mmap = prob.tile, prob.mmap
    g1, w1 = quadrature.gauss_legendre(n_g)
    total = 0.0
    for t in range(mmap.n_tiles):
        for el in tile.elements:
            P = tile.patches[el["patch"]]
            lo, hi = P["lo"], P["hi"]
            pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
            wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
            theta = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
            wgt = np.array([wa * wb * wc for wc in wts[2] for wb in wts[1] for wa in wts[0]]) * np.prod(hi - lo)
            _, J = mmap.tile_map(t, lo + (hi - lo) * theta, ctrl)
            total += np.sum(wgt * np.abs(np.linalg.det(J)))
    return total


def volume_gradient_complex_step(prob, coords, h=1e-30, t_h=None):
    """dV/dP for the listed (control point, component) pairs; only the tiles whose span uses the
    control point change."""
    from .adjoint import tiles_of_control_point
    t_h = tables.volume_table(prob.tile, prob.q) if t_h is None else t_h
    ctrl0 = prob.mmap.macro.ctrl
    out = []
    for k, p in coords:
        c = ctrl0.astype(np.complex128).copy()
        c[k, p] += 1j * h
        v = sum(t_h @ node_abs_det(prob.mmap, t, prob.q, c) for t in tiles_of_control_point(prob, k))
        out.append(np.imag(v) / h)
    return np.array(out)


def body_load(prob, b, ctrl=None, F=None):
    """Global load vector (n_points, 3) of the constant body force b (eq. 53, F = 0 term)."""
    F = tables.load_table(prob.tile, prob.q) if F is None else F
    f = np.zeros((prob.n_points, 3))
    for t in range(prob.mmap.n_tiles):
        s = F @ node_abs_det(prob.mmap, t, prob.q, ctrl)          # (n_T,)
        np.add.at(f, prob.gmap[t], s[:, None] * np.asarray(b)[None, :])
    return f
