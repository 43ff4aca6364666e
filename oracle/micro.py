"""The reference tile T^r (eq. 3) as a multipatch of axis-aligned box patches.

Each patch p maps its parameter cube [0,1]^3 affinely onto the box
[lo_p, hi_p] (control points at the Greville abscissae), so that
T^r_p(theta) = lo_p + (hi_p - lo_p) * theta.  Patches are glued by coincident
control points; a control point keeps the id of the first patch that holds it
(patch order as given, within a patch i + n1*(j + n2*k)), ids compacted in
first-seen order.

The sparsity of the table follows eq. 56: the pairs (A, B), A <= B, whose
supports share at least one micro element (positive-measure overlap), sorted
lexicographically -- this sorted order is the row index m of mat[K] (eq. 57).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import bspline


def open_knots(n_elem: int, p: int) -> np.ndarray:
    inner = np.arange(1, n_elem) / n_elem
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


class ReferenceTile:
    def __init__(self, micro, tol: float = 1e-10):
        self.micro = micro
        self.n_patches = micro.degree.shape[0]
        self.patches = []
        points = []     # positions of unique control points
        ids_all = []
        for p in range(self.n_patches):
            deg = tuple(int(v) for v in micro.degree[p])
            ne = tuple(int(v) for v in micro.n_elem[p])
            knots = tuple(open_knots(ne[d], deg[d]) for d in range(3))
            nfun = tuple(ne[d] + deg[d] for d in range(3))
            lo = np.asarray(micro.box_lo[p], dtype=np.float64)
            hi = np.asarray(micro.box_hi[p], dtype=np.float64)
            grev = [np.array([knots[d][i + 1:i + deg[d] + 1].mean() for i in range(nfun[d])])
                    for d in range(3)]
            ids = np.empty(nfun[0] * nfun[1] * nfun[2], dtype=np.int64)
            for k in range(nfun[2]):
                for j in range(nfun[1]):
                    for i in range(nfun[0]):
                        x = lo + (hi - lo) * np.array([grev[0][i], grev[1][j], grev[2][k]])
                        found = -1
                        for a, y in enumerate(points):
                            if np.max(np.abs(x - y)) < tol:
                                found = a
                                break
                        if found < 0:
                            found = len(points)
                            points.append(x)
                        ids[i + nfun[0] * (j + nfun[1] * k)] = found
            self.patches.append(dict(degree=deg, n_elem=ne, knots=knots, nfun=nfun, lo=lo, hi=hi, ids=ids))
            ids_all.append(ids)
        self.points = np.array(points)          # (n_T, 3) control-point positions t_i of eq. 3
        self.n_T = len(points)
        self._build_elements()
        self._build_pairs()
        self._build_faces(tol)

    # micro elements and their active functions -------------------------------------------
    def _build_elements(self):
        self.elements = []   # dicts: patch, index (e1,e2,e3), theta box, active local ids
        for p, P in enumerate(self.patches):
            ne, deg, nfun = P["n_elem"], P["degree"], P["nfun"]
            for e3, e2, e1 in itertools.product(range(ne[2]), range(ne[1]), range(ne[0])):
                e = (e1, e2, e3)
                th_lo = np.array([e[d] / ne[d] for d in range(3)])
                th_hi = np.array([(e[d] + 1) / ne[d] for d in range(3)])
                # open uniform knots: element e supports patch functions e .. e+deg per direction
                act = [list(range(e[d], e[d] + deg[d] + 1)) for d in range(3)]
                loc = [(a1, a2, a3) for a3 in act[2] for a2 in act[1] for a1 in act[0]]
                glob = [int(P["ids"][a1 + nfun[0] * (a2 + nfun[1] * a3)]) for (a1, a2, a3) in loc]
                self.elements.append(dict(patch=p, e=e, th_lo=th_lo, th_hi=th_hi, loc=loc, ids=glob))

    def _build_pairs(self):
        pairs = set()
        for el in self.elements:
            for A in el["ids"]:
                for B in el["ids"]:
                    if A <= B:
                        pairs.add((A, B))
        self.pairs = np.array(sorted(pairs), dtype=np.int64)      # I_coo, eq. 56
        self.n_nz = len(self.pairs)
        self.pair_index = {(int(a), int(b)): m for m, (a, b) in enumerate(self.pairs)}
        nb = [set() for _ in range(self.n_T)]
        for A, B in self.pairs:
            nb[A].add(int(B))
            nb[B].add(int(A))
        self.neighbours = [sorted(s) for s in nb]

    def _build_faces(self, tol):
        """Local ids on the six faces of [0,1]^3: faces[2*d + s] for xi_d = s."""
        self.faces = []
        for d in range(3):
            for s in (0.0, 1.0):
                on = [a for a in range(self.n_T) if abs(self.points[a, d] - s) < tol]
                # order by the two in-face coordinates so that opposite faces match one to one
                od = [k for k in range(3) if k != d]
                on.sort(key=lambda a: (round(self.points[a, od[1]] / tol), round(self.points[a, od[0]] / tol)))
                self.faces.append(np.array(on, dtype=np.int64))

    # basis evaluation on one patch ----------------------------------------------------------
    def patch_basis(self, p: int, theta: np.ndarray):
        """Values R_a(theta) and theta-gradients of every function of patch p.

        Returns (vals (n, nf), grads (n, nf, 3)), functions ordered a1 + n1*(a2 + n2*a3).
        """
        P = self.patches[p]
        B = [bspline.basis(P["knots"][d], P["degree"][d], theta[:, d]) for d in range(3)]
        D = [bspline.basis_deriv(P["knots"][d], P["degree"][d], theta[:, d]) for d in range(3)]
        n = theta.shape[0]
        vals = np.einsum("pi,pj,pk->pkji", B[0], B[1], B[2]).reshape(n, -1)
        g0 = np.einsum("pi,pj,pk->pkji", D[0], B[1], B[2]).reshape(n, -1)
        g1 = np.einsum("pi,pj,pk->pkji", B[0], D[1], B[2]).reshape(n, -1)
        g2 = np.einsum("pi,pj,pk->pkji", B[0], B[1], D[2]).reshape(n, -1)
        return vals, np.stack([g0, g1, g2], axis=2)

    def counts(self):
        n_ordered = 2 * self.n_nz - self.n_T
        return dict(n_T=self.n_T, n_nz=self.n_nz, n_ordered=n_ordered, n_elements=len(self.elements))
