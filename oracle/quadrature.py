"""Gauss-Legendre rules and the tensor Lagrange basis used as projection space.

The interpolation nodes of degree q are the q+1 Gauss-Legendre points on [0,1]
(reading of eq. 20-24: interpolation at these nodes equals the discrete L2
projection onto Q_q with a (q+1)-point Gauss rule, since the mass matrix is
integrated exactly).  The basis N_C of eq. 42 is then the tensor Lagrange
basis on those nodes, ordered C = c1 + (q+1)(c2 + (q+1) c3); with a degree per direction
(q1, q2, q3) the same with n_d = q_d + 1 nodes in direction d.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(n: int, a: float = 0.0, b: float = 1.0):
    """n-point Gauss-Legendre nodes and weights on [a, b] (numpy's Golub-Welsch routine)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return a + (b - a) * 0.5 * (x + 1.0), 0.5 * (b - a) * w


def lagrange(nodes, x) -> np.ndarray:
    """l_c(x) = prod_{k != c} (x - x_k)/(x_c - x_k); shape (len(x), len(nodes))."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    L = np.ones((len(x), len(nodes)))
    for c in range(len(nodes)):
        for k in range(len(nodes)):
            if k != c:
                L[:, c] *= (x - nodes[k]) / (nodes[c] - nodes[k])
    return L


def interp_nodes(q: int) -> np.ndarray:
    """The q+1 interpolation nodes on [0,1] (ascending)."""
    return gauss_legendre(q + 1)[0]


def degrees(q):
    """Per-direction degrees (q1, q2, q3) of an isotropic degree q or of a 3-sequence."""
    if np.ndim(q) == 0:
        return (int(q),) * 3
    q = tuple(int(v) for v in q)
    assert len(q) == 3
    return q


def n_nodes(q) -> int:
    """n_pi = (q1+1)(q2+1)(q3+1)."""
    q1, q2, q3 = degrees(q)
    return (q1 + 1) * (q2 + 1) * (q3 + 1)


def tensor_nodes(q) -> np.ndarray:
    """All nodes xi_C of the tensor space Q_(q1,q2,q3), C = c1 + n1 (c2 + n2 c3) with n_d = q_d + 1;
    shape (n_pi, 3).  An integer q is the isotropic space."""
    qd = degrees(q)
    g = [interp_nodes(v) for v in qd]
    n1, n2, n3 = (v + 1 for v in qd)
    out = np.empty((n1 * n2 * n3, 3))
    for c3 in range(n3):
        for c2 in range(n2):
            for c1 in range(n1):
                out[c1 + n1 * (c2 + n2 * c3)] = (g[0][c1], g[1][c2], g[2][c3])
    return out


def tensor_lagrange(q, xi) -> np.ndarray:
    """N_C(xi) = l_c1(xi_1) l_c2(xi_2) l_c3(xi_3) for all C at points xi (n, 3) -> (n, n_pi)."""
    qd = degrees(q)
    xi = np.atleast_2d(xi)
    L = [lagrange(interp_nodes(qd[d]), xi[:, d]) for d in range(3)]
    out = np.einsum("pa,pb,pc->pcba", L[0], L[1], L[2]).reshape(len(xi), n_nodes(qd))
    return out
