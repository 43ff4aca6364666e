"""External work of a uniform traction on a macro face (eq. 29, 33): f_A = int_Gamma R_A t dGamma.

The traction t is a force per unit physical area on the part of the tile boundary lying on
the macro face xi_d = s.  On each micro patch face lying there, x = M^(t)(T^r(theta)) and
dGamma = |dx/dtheta_a x dx/dtheta_b| dtheta_a dtheta_b; the integral is taken by a Gauss
rule per micro element face.
"""
from __future__ import annotations

import numpy as np

from . import quadrature, tables


def face_points(prob, face):
    """Global ids of the control points on macro face `face` = 2 d + s, ascending."""
    d, s = face // 2, face % 2
    mm = prob.mmap
    pts = set()
    for t in range(mm.n_tiles):
        if mm.tile_index(t)[d] != (0 if s == 0 else mm.n_elem[d] - 1):
            continue
        pts.update(int(g) for g in prob.gmap[t, prob.tile.faces[face]])
    return np.array(sorted(pts), dtype=np.int64)


def traction_load(prob, face, traction, ctrl=None, n_g=5):
    d, s = face // 2, face % 2
    ia, ib = [k for k in range(3) if k != d]
    mm, tile = prob.mmap, prob.tile
    f = np.zeros((prob.n_points, 3))
    g1, w1 = quadrature.gauss_legendre(n_g)
    tr = np.asarray(traction, dtype=np.float64)
    for t in range(mm.n_tiles):
        if mm.tile_index(t)[d] != (0 if s == 0 else mm.n_elem[d] - 1):
            continue
        for p, P in enumerate(tile.patches):
            lo, hi = P["lo"], P["hi"]
            if not ((s == 0 and lo[d] == 0.0) or (s == 1 and hi[d] == 1.0)):
                continue
            ne = P["n_elem"]
            for eb in range(ne[ib]):
                for ea in range(ne[ia]):
                    th = np.zeros((n_g * n_g, 3))
                    th[:, d] = float(s)
                    ta = (ea + g1) / ne[ia]
                    tb = (eb + g1) / ne[ib]
                    th[:, ia] = np.tile(ta, n_g)
                    th[:, ib] = np.repeat(tb, n_g)
                    w = np.outer(w1, w1).ravel() / (ne[ia] * ne[ib])
                    xi = lo + (hi - lo) * th
                    _, J = mm.tile_map(t, xi, ctrl)
                    da = J[:, :, ia] * (hi - lo)[ia]
                    db = J[:, :, ib] * (hi - lo)[ib]
                    dA = np.linalg.norm(np.cross(da, db), axis=1) * w
                    vals, _ = tile.patch_basis(p, th)
                    ids = P["ids"]
                    for a in range(vals.shape[1]):
                        r = vals[:, a] @ dA
                        if r != 0.0:
                            f[prob.gmap[t, ids[a]]] += r * tr
    return f


def traction_load_lookup(prob, face, traction, q, ctrl=None, F=None):
    """The traction part of eq. 53: per tile on the macro face xi_d = s, the projected macro
    traction <t_bar>_C2 = t |det I_M| (eq. 87-88) at the face nodes, where on that face
    det I_M = (n x g_a) . g_b = |g_a x g_b| with g_k = dM/dxi_k (the unit normal along the
    contravariant g^d), times the face table: f_A += sum_C2 F_face[A, C2] <t_bar>_C2."""
    d, s = face // 2, face % 2
    ia, ib = [k for k in range(3) if k != d]
    mm, tile = prob.mmap, prob.tile
    F = tables.face_load_table(tile, q, face) if F is None else F
    uv = tables.face_nodes(q, face)
    xi = np.zeros((len(uv), 3))
    xi[:, d] = float(s)
    xi[:, ia], xi[:, ib] = uv[:, 0], uv[:, 1]
    tr = np.asarray(traction, dtype=np.float64)
    f = np.zeros((prob.n_points, 3))
    for t in range(mm.n_tiles):
        if mm.tile_index(t)[d] != (0 if s == 0 else mm.n_elem[d] - 1):
            continue
        _, J = mm.tile_map(t, xi, ctrl)
        area = np.linalg.norm(np.cross(J[:, :, ia], J[:, :, ib]), axis=1)     # |det I_M| at the nodes
        fa = F @ area
        for A in np.nonzero(fa)[0]:
            f[prob.gmap[t, A]] += fa[A] * tr
    return f
