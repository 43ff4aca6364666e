"""Sensitivity of the lookup-form stiffness to the macro control points (Sec. 4.1.2, eq. 69-73).

The quantity differentiated is the quadratic form Q(P) = u^T K_pi(P) u for a fixed
displacement vector u, whose gradient is the internal-work term of eq. 69-70:
dQ/dP = u^T (dK_pi/dP) u.  (With f fixed and u = K^-1 f the compliance C = f^T u
has dC/dP = -u^T (dK/dP) u.)

The oracle takes the derivative by complex-step differentiation (Squire and Trapp
1998): Q(P + i h e_k) is evaluated with complex arithmetic through the same lookup-form
assembly (eq. 50, 58) and dQ/dP_k = Im Q / h, exact to rounding for h ~ 1e-30.
Only tiles whose knot span involves control point k change, so only those are summed.
"""
from __future__ import annotations

import numpy as np

from .assembly import coefficient_block


def tile_quadratic(prob, t, u_pts, ctrl, relative=False):
    """u_t^T K_t u_t for tile t, with the tile's lookup-form blocks (eq. 58); complex-safe.

    relative=True evaluates the same number as v_t^T K_t v_t with v_t = u_t - u_t[local point 0]:
    K_t annihilates translations for any control net (the basis functions sum to one, so their
    derivatives, and every row of the table, sum to zero; eq. 56-57), and the shifted form avoids
    the cancellation of a large rigid-body displacement in floating point."""
    n_nz = prob.T.shape[0]
    Kt = (prob.T.reshape(n_nz, -1) @ coefficient_block(prob.mmap, t, prob.q, prob.lam, prob.mu, ctrl)
          ).reshape(n_nz, 3, 3)
    P = prob.tile.pairs
    g = prob.gmap[t]
    ua, ub = u_pts[g[P[:, 0]]], u_pts[g[P[:, 1]]]
    if relative:
        ua, ub = ua - u_pts[g[0]], ub - u_pts[g[0]]
    w = np.where(P[:, 0] == P[:, 1], 1.0, 2.0)             # upper block and its transpose
    return np.einsum("m,ma,mab,mb->", w, ua, Kt, ub)


def quadratic_form(prob, u, ctrl=None):
    """Q = u^T K u for the whole structure (u: (n_points, 3) or flat)."""
    ctrl = prob.mmap.macro.ctrl if ctrl is None else ctrl
    u_pts = np.asarray(u).reshape(-1, 3)
    return sum(tile_quadratic(prob, t, u_pts, ctrl) for t in range(prob.mmap.n_tiles))


def tiles_of_control_point(prob, k):
    """Tiles whose span uses control point k (index i + n1 (j + n2 l))."""
    mm = prob.mmap
    n1, n2, _ = mm.macro.n_ctrl_dir
    idx = (k % n1, (k // n1) % n2, k // (n1 * n2))
    out = []
    for t in range(mm.n_tiles):
        ti = mm.tile_index(t)
        ok = True
        for d in range(3):
            p = mm.degree[d]
            lo, _ = mm.spans[d][ti[d]]
            span = np.searchsorted(mm.knots[d], lo, side="right") - 1   # knot index k of [t_k, t_k+1)
            if not (span - p <= idx[d] <= span):
                ok = False
                break
        if ok:
            out.append(t)
    return out


def gradient_complex_step(prob, u, coords, h=1e-30, relative=False):
    """dQ/dP for the listed (control point, component) pairs by complex step (relative: see
    tile_quadratic)."""
    ctrl0 = prob.mmap.macro.ctrl
    u_pts = np.asarray(u).reshape(-1, 3)
    out = []
    for k, p in coords:
        c = ctrl0.astype(np.complex128).copy()
        c[k, p] += 1j * h
        q = sum(tile_quadratic(prob, t, u_pts, c, relative) for t in tiles_of_control_point(prob, k))
        out.append(np.imag(q) / h)
    return np.array(out)


def gradient_central_fd(prob, u, coords, h=1e-6):
    """The same derivatives by central differences (sanity check of the complex step)."""
    ctrl0 = prob.mmap.macro.ctrl
    u_pts = np.asarray(u).reshape(-1, 3)
    out = []
    for k, p in coords:
        ts = tiles_of_control_point(prob, k)
        cp, cm = ctrl0.copy(), ctrl0.copy()
        cp[k, p] += h
        cm[k, p] -= h
        qp = sum(tile_quadratic(prob, t, u_pts, cp) for t in ts)
        qm = sum(tile_quadratic(prob, t, u_pts, cm) for t in ts)
        out.append((qp - qm) / (2 * h))
    return np.array(out)


def gradient_all(prob, u, h=1e-30):
    """dQ/dP for every control point and component, (n_ctrl, 3), by complex step (small cases)."""
    n = prob.mmap.macro.ctrl.shape[0]
    g = gradient_complex_step(prob, u, [(k, p) for k in range(n) for p in range(3)], h)
    return g.reshape(n, 3)
