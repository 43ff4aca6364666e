"""Stiffness lookup table mat[K] (eq. 49-52, 56-57) by Gauss quadrature over micro elements.

  T[m, C, i, j] = int_{Omega_T} d/dxi_i (R_A o T^r^-1) * d/dxi_j (R_B o T^r^-1) * N_C dxi,

for every pair m = (A, B) of I_coo (eq. 56).  Each micro element is a box of a
patch; on it xi = lo + (hi - lo) theta, so d/dxi_i = (1/(hi-lo)_i) d/dtheta_i and
dxi = prod(hi - lo) dtheta.  The integrand is a polynomial on the element, of
degree at most 2 p_T + q per direction, so an n_g-point rule with
2 n_g - 1 >= 2 p_T + q integrates it exactly ("accurate enough numerical
integration", eq. 52).
"""
from __future__ import annotations

import numpy as np

from . import quadrature


def default_gauss_points(p_T: int, q: int) -> int:
    return (2 * p_T + q + 2) // 2


def build_table(tile, q: int, n_g: int | None = None) -> np.ndarray:
    """mat[K] as an array (n_nz, (q+1)^3, 3, 3)."""
    p_T = max(max(P["degree"]) for P in tile.patches)
    n_g = n_g or default_gauss_points(p_T, max(quadrature.degrees(q)))
    n_pi = quadrature.n_nodes(q)
    T = np.zeros((tile.n_nz, n_pi, 3, 3))
    g1, w1 = quadrature.gauss_legendre(n_g)
    for el in tile.elements:
        P = tile.patches[el["patch"]]
        lo, hi = P["lo"], P["hi"]
        # element Gauss points in the patch parameter theta
        pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
        wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
        theta = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
        wgt = np.array([wa * wb * wc for wc in wts[2] for wb in wts[1] for wa in wts[0]])
        wgt = wgt * np.prod(hi - lo)                    # |det J_{T^r}| for the affine patch
        xi = lo + (hi - lo) * theta
        _, grads = tile.patch_basis(el["patch"], theta)  # (g, nf, 3) in theta
        nf = P["nfun"]
        cols = [a1 + nf[0] * (a2 + nf[1] * a3) for (a1, a2, a3) in el["loc"]]
        dphi = grads[:, cols, :] / (hi - lo)            # (g, 27, 3) d/dxi
        NC = quadrature.tensor_lagrange(q, xi)          # (g, n_pi)
        # local contribution Tloc[a, b, C, i, j] = sum_g w dphi[g,a,i] dphi[g,b,j] N_C
        Tloc = np.einsum("g,gai,gbj,gc->abcij", wgt, dphi, dphi, NC, optimize=True)
        ids = el["ids"]
        for a, A in enumerate(ids):
            for b, B in enumerate(ids):
                if A <= B:
                    T[tile.pair_index[(A, B)]] += Tloc[a, b]
    return T


def volume_table(tile, q: int, n_g: int | None = None) -> np.ndarray:
    """t^h of eq. 18 for the projection basis N_C: t_C = int_{Omega_T} N_C dxi."""
    p_T = max(max(P["degree"]) for P in tile.patches)
    n_g = n_g or default_gauss_points(p_T, max(quadrature.degrees(q)))
    g1, w1 = quadrature.gauss_legendre(n_g)
    t = np.zeros(quadrature.n_nodes(q))
    for el in tile.elements:
        P = tile.patches[el["patch"]]
        lo, hi = P["lo"], P["hi"]
        pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
        wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
        theta = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
        wgt = np.array([wa * wb * wc for wc in wts[2] for wb in wts[1] for wa in wts[0]]) * np.prod(hi - lo)
        t += wgt @ quadrature.tensor_lagrange(q, lo + (hi - lo) * theta)
    return t


def load_table(tile, q: int, n_g: int | None = None) -> np.ndarray:
    """The body-force part of the load lookup table (eq. 54-55, F = 0):
    F[A, C] = int_{Omega_T} (R_A o T^r^-1) N_C dxi, shape (n_T, (q+1)^3), by the same element
    quadrature as the stiffness table (the integrand has degree <= p_T + q per direction)."""
    p_T = max(max(P["degree"]) for P in tile.patches)
    n_g = n_g or default_gauss_points(p_T, max(quadrature.degrees(q)))
    g1, w1 = quadrature.gauss_legendre(n_g)
    F = np.zeros((tile.n_T, quadrature.n_nodes(q)))
    for el in tile.elements:
        P = tile.patches[el["patch"]]
        lo, hi = P["lo"], P["hi"]
        pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
        wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
        theta = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
        wgt = np.array([wa * wb * wc for wc in wts[2] for wb in wts[1] for wa in wts[0]]) * np.prod(hi - lo)
        vals, _ = tile.patch_basis(el["patch"], theta)
        nf = P["nfun"]
        cols = [a1 + nf[0] * (a2 + nf[1] * a3) for (a1, a2, a3) in el["loc"]]
        NC = quadrature.tensor_lagrange(q, lo + (hi - lo) * theta)
        Floc = np.einsum("g,ga,gc->ac", wgt, vals[:, cols], NC)
        for a, A in enumerate(el["ids"]):
            F[A] += Floc[a]
    return F



def _face_degrees(q, face: int):
    d = face // 2
    ia, ib = [k for k in range(3) if k != d]
    qd = quadrature.degrees(q)
    return qd[ia], qd[ib]


def face_nodes(q, face: int = 0) -> np.ndarray:
    """The (q_a+1)(q_b+1) nodes of the face projection space of `face`, C2 = c_a + (q_a+1) c_b in
    the two in-face directions a < b; shape (n, 2)."""
    qa, qb = _face_degrees(q, face)
    ga, gb = quadrature.interp_nodes(qa), quadrature.interp_nodes(qb)
    return np.array([(ga[ca], gb[cb]) for cb in range(qb + 1) for ca in range(qa + 1)])


def face_lagrange(q, uv, face: int = 0) -> np.ndarray:
    """N_C2(u, v) = l_ca(u) l_cb(v) at points uv (n, 2) of `face` -> (n, (q_a+1)(q_b+1))."""
    qa, qb = _face_degrees(q, face)
    uv = np.atleast_2d(uv)
    La = quadrature.lagrange(quadrature.interp_nodes(qa), uv[:, 0])
    Lb = quadrature.lagrange(quadrature.interp_nodes(qb), uv[:, 1])
    return np.einsum("pa,pb->pba", La, Lb).reshape(len(uv), -1)


def face_load_table(tile, q: int, face: int, n_g: int | None = None) -> np.ndarray:
    """The traction part of the load lookup table (eq. 54-55, F = face + 1):
    F_face[A, C2] = int over the part of the tile boundary on the cube face xi_d = s (face = 2 d + s)
    of (R_A o T^r^-1) N_C2 dGamma_T, with N_C2 the degree-q Lagrange basis of the face's own
    Gauss-Legendre nodes in its two in-face coordinates (the reading of the node set I_F for this
    basis).  Integrated per micro element face by Gauss quadrature (exact: polynomial integrand);
    shape (n_T, (q+1)^2)."""
    d, s = face // 2, face % 2
    ia, ib = [k for k in range(3) if k != d]
    p_T = max(max(P["degree"]) for P in tile.patches)
    n_g = n_g or default_gauss_points(p_T, max(quadrature.degrees(q)))
    g1, w1 = quadrature.gauss_legendre(n_g)
    qa, qb = _face_degrees(q, face)
    F = np.zeros((tile.n_T, (qa + 1) * (qb + 1)))
    for p, P in enumerate(tile.patches):
        lo, hi = P["lo"], P["hi"]
        if not ((s == 0 and lo[d] == 0.0) or (s == 1 and hi[d] == 1.0)):
            continue
        ne = P["n_elem"]
        for eb in range(ne[ib]):
            for ea in range(ne[ia]):
                th = np.zeros((n_g * n_g, 3))
                th[:, d] = float(s)
                th[:, ia] = np.tile((ea + g1) / ne[ia], n_g)
                th[:, ib] = np.repeat((eb + g1) / ne[ib], n_g)
                w = np.outer(w1, w1).ravel() / (ne[ia] * ne[ib]) * (hi - lo)[ia] * (hi - lo)[ib]
                xi = lo + (hi - lo) * th
                vals, _ = tile.patch_basis(p, th)
                N2 = face_lagrange(q, xi[:, [ia, ib]], face)
                Floc = np.einsum("g,ga,gc->ac", w, vals, N2)
                for a, A in enumerate(P["ids"]):
                    F[A] += Floc[a]
    return F
