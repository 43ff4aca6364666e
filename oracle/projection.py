"""Projection error of the macro field and the choice of the projection degree (Sec. 3.2.2, eq. 47-48;
Sec. 3.3, eq. 59, 65) -- test infrastructure.

E_proj = max over tiles and sample points xi of ||A_bar(xi) - Pi A_bar(xi)||_F / ||A_bar(xi)||_F
(eq. 59), the Frobenius norm over the 81 components (i, j, alpha, beta); Pi is the interpolant at the
(q+1)^3 Gauss-Legendre nodes (the projection reading used throughout), or the L2 projection onto Q_q
of eq. 20-24 (l2_coefficients).  The sample set is the uniform interior grid xi_s = (s + 1/2) / n_s
per direction ("a simple sampling-based approach").  The degree is raised from q0 until
E_proj <= tol (eq. 65).
"""
from __future__ import annotations

import numpy as np

from . import pullback, quadrature
from .macro import MacroMap


def sample_points(n_s: int) -> np.ndarray:
    g = (np.arange(n_s) + 0.5) / n_s
    return np.array([(a, b, c) for c in g for b in g for a in g])


def tensor_gauss(n: int):
    """The n^3-point tensor Gauss-Legendre rule on [0,1]^3: points (n^3, 3) in the node order
    g1 + n (g2 + n g3), and weights (n^3,)."""
    x, w = quadrature.gauss_legendre(n)
    pts = np.array([(x[a], x[b], x[c]) for c in range(n) for b in range(n) for a in range(n)])
    wts = np.array([w[a] * w[b] * w[c] for c in range(n) for b in range(n) for a in range(n)])
    return pts, wts


def l2_coefficients(mmap: MacroMap, t: int, q: int, lam: float, mu: float, n_g: int, ctrl=None):
    """The L2 projection of tile t's macro field onto Q_q (eq. 20-24): the coefficients a (per node C
    of the degree-q Lagrange basis N_C, 81 components each) minimising the L2 norm of
    A_bar - sum_C a_C N_C solve the normal equations M a = b, with the mass matrix M_CD = int N_C N_D
    (integrated exactly: a rule of 2q+2 points per direction, for its degree-2q integrand) and the
    load b_C = int N_C A_bar, integrated by the n_g-point Gauss rule per direction.
    Returns (n_pi, 81) in the layout of the nodal values (n_pi, i, j, alpha, beta)."""
    xm, wm = tensor_gauss(2 * max(quadrature.degrees(q)) + 2)
    Nm = quadrature.tensor_lagrange(q, xm)                       # (n_m, n_pi)
    M = Nm.T @ (wm[:, None] * Nm)
    xg, wg = tensor_gauss(n_g)
    _, J = mmap.tile_map(t, xg, ctrl)
    A = pullback.macro_field(J, lam, mu).reshape(len(xg), 81)   # the field at the quadrature points
    Ng = quadrature.tensor_lagrange(q, xg)
    b = Ng.T @ (wg[:, None] * A)                                  # (n_pi, 81)
    return np.linalg.solve(M, b)


def tile_projection_error(mmap: MacroMap, t: int, q: int, lam: float, mu: float, n_s: int = 5, ctrl=None,
                          points=None, n_gauss: int = 0):
    """Largest relative Frobenius error of the projected field over the samples of tile t; the
    interpolant at the nodes, or (n_gauss > 0) the L2 projection with an n_gauss-point load rule."""
    xi = sample_points(n_s) if points is None else points
    _, Js = mmap.tile_map(t, xi, ctrl)
    exact = pullback.macro_field(Js, lam, mu).reshape(len(xi), 81)
    if n_gauss > 0:
        coef = l2_coefficients(mmap, t, q, lam, mu, n_gauss, ctrl)
    else:
        _, Jn = mmap.tile_map(t, quadrature.tensor_nodes(q), ctrl)
        coef = pullback.macro_field(Jn, lam, mu).reshape(-1, 81)
    approx = quadrature.tensor_lagrange(q, xi) @ coef
    return np.max(np.linalg.norm(exact - approx, axis=1) / np.linalg.norm(exact, axis=1))


def projection_error(macro, q: int, E: float = 1.0, nu: float = 0.3, n_s: int = 5, ctrl=None, n_gauss: int = 0):
    """(per-tile errors, E_proj) of eq. 59 (interpolant, or L2 projection with n_gauss > 0)."""
    lam, mu = pullback.lame(E, nu)
    mmap = MacroMap(macro)
    e = np.array([tile_projection_error(mmap, t, q, lam, mu, n_s, ctrl, n_gauss=n_gauss)
                  for t in range(mmap.n_tiles)])
    return e, e.max()


BAND = 1e-9      # errors within this relative band are equal (see select_degrees)


def meets(err: float, tol: float) -> bool:
    """E_proj <= tol, with an error within a relative BAND above tol counted as meeting it."""
    return err <= tol * (1.0 + BAND)


def select_degree(macro, tol: float, q0: int, q_max: int, **kw):
    """Smallest q >= q0 with E_proj <= tol (eq. 65; within the relative BAND), or q_max."""
    for q in range(q0, q_max + 1):
        if meets(projection_error(macro, q, **kw)[1], tol):
            return q
    return q_max


def select_degrees(macro, tol: float, q_init, q_max: int = 7, **kw):
    """A degree per direction (the anisotropic projection space of Sec. 3.3.4): from q_init (the
    macro map's degrees), enrich while E_proj > tol, each step raising the one direction whose
    increase lowers E_proj most; then coarsen while possible, each step lowering the direction whose
    decrease keeps E_proj lowest, as long as it stays <= tol.  Errors within a relative 1e-9 (BAND) of
    each other are ties, which go to the lowest direction, and an error within BAND above tol meets
    it: rounding differences between implementations must not decide the path.
    Returns (degrees, E_proj)."""
    q = list(quadrature.degrees(q_init))
    err = projection_error(macro, tuple(q), **kw)[1]
    while not meets(err, tol):
        best = None
        for d in range(3):
            if q[d] >= q_max:
                continue
            c = q.copy()
            c[d] += 1
            e = projection_error(macro, tuple(c), **kw)[1]
            if best is None or e < best[0] * (1.0 - BAND):   # within the band: a tie, the lower direction
                best = (e, c)
        if best is None:
            break
        err, q = best
    while True:
        best = None
        for d in range(3):
            if q[d] == 0:
                continue
            c = q.copy()
            c[d] -= 1
            e = projection_error(macro, tuple(c), **kw)[1]
            if meets(e, tol) and (best is None or e < best[0] * (1.0 - BAND)):
                best = (e, c)
        if best is None:
            break
        err, q = best
    return tuple(q), err
