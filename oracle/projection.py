"""Projection error of the macro field and the choice of the projection degree (Sec. 3.2.2, eq. 47-48;
Sec. 3.3, eq. 59, 65) -- test infrastructure.

E_proj = max over tiles and sample points xi of ||A_bar(xi) - Pi A_bar(xi)||_F / ||A_bar(xi)||_F
(eq. 59), the Frobenius norm over the 81 components (i, j, alpha, beta); Pi is the interpolant at the
(q+1)^3 Gauss-Legendre nodes (the projection reading used throughout).  The sample set is the uniform
interior grid xi_s = (s + 1/2) / n_s per direction ("a simple sampling-based approach").  The degree
is raised from q0 until E_proj <= tol (eq. 65).
"""
from __future__ import annotations

import numpy as np

from . import pullback, quadrature
from .macro import MacroMap


def sample_points(n_s: int) -> np.ndarray:
    g = (np.arange(n_s) + 0.5) / n_s
    return np.array([(a, b, c) for c in g for b in g for a in g])


def tile_projection_error(mmap: MacroMap, t: int, q: int, lam: float, mu: float, n_s: int = 5, ctrl=None,
                          points=None):
    xi = sample_points(n_s) if points is None else points
    _, Js = mmap.tile_map(t, xi, ctrl)
    exact = pullback.macro_field(Js, lam, mu).reshape(len(xi), 81)
    _, Jn = mmap.tile_map(t, quadrature.tensor_nodes(q), ctrl)
    nodes = pullback.macro_field(Jn, lam, mu).reshape(-1, 81)
    interp = quadrature.tensor_lagrange(q, xi) @ nodes
    return np.max(np.linalg.norm(exact - interp, axis=1) / np.linalg.norm(exact, axis=1))


def projection_error(macro, q: int, E: float = 1.0, nu: float = 0.3, n_s: int = 5, ctrl=None):
    """(per-tile errors, E_proj) of eq. 59."""
    lam, mu = pullback.lame(E, nu)
    mmap = MacroMap(macro)
    e = np.array([tile_projection_error(mmap, t, q, lam, mu, n_s, ctrl) for t in range(mmap.n_tiles)])
    return e, e.max()


def select_degree(macro, tol: float, q0: int, q_max: int, **kw):
    """Smallest q >= q0 with E_proj <= tol (eq. 65), or q_max."""
    for q in range(q0, q_max + 1):
        if projection_error(macro, q, **kw)[1] <= tol:
            return q
    return q_max
