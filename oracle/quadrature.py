"""Gauss-Legendre rules and the tensor Lagrange basis used as projection space.

The interpolation nodes of degree q are the q+1 Gauss-Legendre points on [0,1]
(reading of eq. 20-24: interpolation at these nodes equals the discrete L2
projection onto Q_q with a (q+1)-point Gauss rule, since the mass matrix is
integrated exactly).  The basis N_C of eq. 42 is then the tensor Lagrange
basis on those nodes, ordered C = c1 + (q+1)(c2 + (q+1) c3).
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


def tensor_nodes(q: int) -> np.ndarray:
    """All (q+1)^3 nodes xi_C, C = c1 + (q+1)(c2 + (q+1) c3); shape ((q+1)^3, 3)."""
    g = interp_nodes(q)
    n = q + 1
    out = np.empty((n ** 3, 3))
    for c3 in range(n):
        for c2 in range(n):
            for c1 in range(n):
                out[c1 + n * (c2 + n * c3)] = (g[c1], g[c2], g[c3])
    return out


def tensor_lagrange(q: int, xi) -> np.ndarray:
    """N_C(xi) for all C at points xi (n, 3) -> (n, (q+1)^3)."""
    g = interp_nodes(q)
    xi = np.atleast_2d(xi)
    L = [lagrange(g, xi[:, d]) for d in range(3)]
    n = q + 1
    out = np.einsum("pa,pb,pc->pcba", L[0], L[1], L[2]).reshape(len(xi), n ** 3)
    return out
