"""Tile maps of the macro B-spline (eq. 4-8).

Tile t = (ix, iy, iz), linear index ix + nx*(iy + ny*iz), is the knot-span box
[u0_x, u1_x] x [u0_y, u1_y] x [u0_z, u1_z]; its map on [0,1]^3 is
M^(t)(xi) = M(u0 + (u1 - u0) xi), which is the Bezier element of eq. 7-8
evaluated without forming the extraction explicitly.
"""
from __future__ import annotations

import numpy as np

from . import bspline


class MacroMap:
    def __init__(self, macro):
        self.macro = macro
        self.degree = tuple(macro.degree)
        self.knots = tuple(np.asarray(k, dtype=np.float64) for k in macro.knots)
        self.spans = [bspline.spans(k) for k in self.knots]
        self.n_elem = tuple(len(s) for s in self.spans)
        self.n_tiles = int(np.prod(self.n_elem))

    def tile_index(self, t: int):
        nx, ny, _ = self.n_elem
        return t % nx, (t // nx) % ny, t // (nx * ny)

    def tile_box(self, t: int):
        idx = self.tile_index(t)
        lo = np.array([self.spans[d][idx[d], 0] for d in range(3)])
        hi = np.array([self.spans[d][idx[d], 1] for d in range(3)])
        return lo, hi

    def tile_map(self, t: int, xi: np.ndarray, ctrl: np.ndarray | None = None):
        """x = M^(t)(xi) and J^(t)(xi)[p, i] = d x_p / d xi_i at points xi (n, 3)."""
        ctrl = self.macro.ctrl if ctrl is None else ctrl
        lo, hi = self.tile_box(t)
        u = lo + (hi - lo) * np.atleast_2d(xi)
        x, J = bspline.volume_eval(self.knots, self.degree, ctrl, u)
        return x, J * (hi - lo)[None, None, :]
