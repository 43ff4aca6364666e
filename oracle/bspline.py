"""B-spline basis functions by the Cox-de Boor recursion (eq. 1-4 build splines on them).

Plain definitions, evaluated for *all* n basis functions of a knot vector at once,
with the convention 0/0 = 0.  The last non-empty knot span is closed on the right
so that u = t_end is evaluated as a limit from inside.
"""
from __future__ import annotations

import numpy as np


def _degree0(knots: np.ndarray, u: np.ndarray) -> np.ndarray:
    """N_{i,0}(u) = 1 on [t_i, t_{i+1}), for every i; shape (len(u), len(knots)-1)."""
    t = knots
    m = len(t) - 1
    N = np.zeros((len(u), m))
    last = max(i for i in range(m) if t[i + 1] > t[i])  # last non-empty span
    for i in range(m):
        if t[i + 1] > t[i]:
            inside = (u >= t[i]) & (u < t[i + 1])
            if i == last:
                inside |= (u == t[i + 1])
            N[:, i] = inside
    return N


def _ratio(num, den):
    return np.where(den != 0.0, num / np.where(den != 0.0, den, 1.0), 0.0)


def basis(knots, p: int, u) -> np.ndarray:
    """All degree-p basis functions at the points u: array (len(u), n), n = len(knots)-p-1."""
    t = np.asarray(knots, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    N = _degree0(t, u)
    for k in range(1, p + 1):
        nk = len(t) - k - 1
        new = np.zeros((len(u), nk))
        for i in range(nk):
            left = _ratio(u - t[i], t[i + k] - t[i]) * N[:, i]
            right = _ratio(t[i + k + 1] - u, t[i + k + 1] - t[i + 1]) * N[:, i + 1]
            new[:, i] = left + right
        N = new
    return N


def basis_deriv(knots, p: int, u) -> np.ndarray:
    """First derivatives dN_{i,p}/du at u, from the degree-(p-1) functions:
    N'_{i,p} = p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}."""
    t = np.asarray(knots, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    n = len(t) - p - 1
    if p == 0:
        return np.zeros((len(u), n))
    Nm = basis(t, p - 1, u)  # (len(u), n+1)
    d = np.zeros((len(u), n))
    for i in range(n):
        a = p / (t[i + p] - t[i]) if t[i + p] != t[i] else 0.0
        b = p / (t[i + p + 1] - t[i + 1]) if t[i + p + 1] != t[i + 1] else 0.0
        d[:, i] = a * Nm[:, i] - b * Nm[:, i + 1]
    return d


def spans(knots) -> np.ndarray:
    """Non-empty knot spans [t_k, t_{k+1}] as an (n_elem, 2) array, in increasing order."""
    t = np.asarray(knots, dtype=np.float64)
    out = [(t[i], t[i + 1]) for i in range(len(t) - 1) if t[i + 1] > t[i]]
    return np.array(out, dtype=np.float64)


def volume_eval(knots3, degree3, ctrl, u3):
    """Trivariate spline value and parametric Jacobian at points u3 (n, 3) (eq. 2, 4).

    ctrl row i + n1*(j + n2*k) holds control point (i, j, k).  Returns
    x (n, 3) and dx/du (n, 3, 3) with [p, d] = d x_p / d u_d.
    """
    u3 = np.atleast_2d(np.asarray(u3, dtype=np.float64))
    B = [basis(knots3[d], degree3[d], u3[:, d]) for d in range(3)]
    D = [basis_deriv(knots3[d], degree3[d], u3[:, d]) for d in range(3)]
    n1, n2, n3 = (b.shape[1] for b in B)
    net = ctrl.reshape(n3, n2, n1, 3)  # net[k, j, i] = ctrl[i + n1*(j + n2*k)]
    x = np.einsum("ni,nj,nk,kjip->np", B[0], B[1], B[2], net)
    J = np.empty((u3.shape[0], 3, 3), dtype=np.result_type(ctrl, B[0]))   # complex-safe
    J[:, :, 0] = np.einsum("ni,nj,nk,kjip->np", D[0], B[1], B[2], net)
    J[:, :, 1] = np.einsum("ni,nj,nk,kjip->np", B[0], D[1], B[2], net)
    J[:, :, 2] = np.einsum("ni,nj,nk,kjip->np", B[0], B[1], D[2], net)
    return x, J
