"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *describes* inputs: macro control nets and knot vectors, the
micro-tile patch boxes, strut-width fields and random vectors.  It contains none
of the assembly method's arithmetic (no basis evaluation, no quadrature, no
pullback, no numbering), so both implementations can consume it without sharing
any of the computation they are compared on.

Geometry recipes (all lengths in tile units):

* micro tile -- the 3D cross cell: a central cube [0.5-w/2, 0.5+w/2]^3 and six
  struts of width w reaching the faces of [0,1]^3; 7 axis-aligned box patches
  ordered [centre, -x, +x, -y, +y, -z, +z], each a degree-2 B-spline with n_e
  uniform elements per direction (the reference tile of Sec. 2.2.2, eq. 3).
* perturbed cube -- one cubic Bezier cube, control points {0,1/3,2/3,1}^3 plus
  U(-amp, amp)^3 noise, refined by knot insertion at 1/2 in every direction so
  that it has 2x2x2 elements (tiles) with unchanged geometry.
* twisted beam -- [0,nx]x[-ny/2,ny/2]x[-nz/2,nz/2], the cross-section rotated
  about x by (pi/2) x/nx; degree-3 open uniform B-spline with one element per
  tile; control points = the twist applied to the Greville points.
* quarter arc -- [0,20]x[0,10]x[0,10] (generally nx x ny x nz) bent by
  phi=(pi/2) x/nx, R = R_c + (y - ny/2), R_c = 2 nx/pi, point (R cos phi,
  R sin phi, z), applied at the Greville points.
* cantilever plate -- the box [0,nx]x[0,ny]x[0,nz] (affine Greville net).
* width field -- w_t = 0.275 + 0.125 sin(2 pi x+p1) sin(2 pi y+p2) sin(2 pi z+p3)
  at normalised tile centres, phases p_k ~ U(0, 2 pi) from the seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "MicroDesc", "MacroDesc", "micro_cross", "macro_perturbed_cube", "macro_twisted_beam",
    "macro_quarter_arc", "macro_cantilever", "macro_affine_box", "width_field", "rng",
    "WORKLOADS", "workload",
]

PATCH_NAMES = ("centre", "-x", "+x", "-y", "+y", "-z", "+z")


def rng(seed: int) -> np.random.Generator:
    """Host PCG64 generator used for every seeded draw."""
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class MicroDesc:
    """Reference tile as a list of axis-aligned box patches (degree, elements, box)."""
    degree: np.ndarray      # (n_patches, 3) int32
    n_elem: np.ndarray      # (n_patches, 3) int32
    box_lo: np.ndarray      # (n_patches, 3) float64
    box_hi: np.ndarray      # (n_patches, 3) float64
    width: float = 0.3

    @property
    def n_patches(self) -> int:
        return int(self.degree.shape[0])


@dataclass
class MacroDesc:
    """Trivariate B-spline macro map: degrees, open knot vectors, control net.

    ``ctrl`` has shape (n1*n2*n3, 3), control point (i, j, k) stored at row
    i + n1*(j + n2*k).
    """
    degree: tuple
    knots: tuple            # three 1-D float64 arrays
    ctrl: np.ndarray        # (n_ctrl, 3) float64
    name: str = ""

    @property
    def n_ctrl_dir(self) -> tuple:
        return tuple(len(self.knots[d]) - self.degree[d] - 1 for d in range(3))

    @property
    def n_elem(self) -> tuple:
        return tuple(len(np.unique(self.knots[d])) - 1 for d in range(3))

    @property
    def n_tiles(self) -> int:
        e = self.n_elem
        return e[0] * e[1] * e[2]


def micro_cross(n_e: int, width: float = 0.3, degree: int = 2) -> MicroDesc:
    """The 3D cross lattice cell (7 box patches) with strut width ``width``."""
    c0, c1 = 0.5 - 0.5 * width, 0.5 + 0.5 * width
    mid = (c0, c1)
    boxes = [
        ((c0, c1), mid, mid),          # centre
        ((0.0, c0), mid, mid),         # -x
        ((c1, 1.0), mid, mid),         # +x
        (mid, (0.0, c0), mid),         # -y
        (mid, (c1, 1.0), mid),         # +y
        (mid, mid, (0.0, c0)),         # -z
        (mid, mid, (c1, 1.0)),         # +z
    ]
    lo = np.array([[b[d][0] for d in range(3)] for b in boxes], dtype=np.float64)
    hi = np.array([[b[d][1] for d in range(3)] for b in boxes], dtype=np.float64)
    n = len(boxes)
    return MicroDesc(degree=np.full((n, 3), degree, np.int32), n_elem=np.full((n, 3), n_e, np.int32),
                     box_lo=lo, box_hi=hi, width=float(width))


def open_uniform_knots(n_elem: int, degree: int) -> np.ndarray:
    inner = np.arange(1, n_elem, dtype=np.float64) / n_elem
    return np.concatenate([np.zeros(degree + 1), inner, np.ones(degree + 1)])


def greville(knots: np.ndarray, degree: int) -> np.ndarray:
    """Greville abscissae (knot averages) -- where an affine spline puts its control points."""
    n = len(knots) - degree - 1
    return np.array([knots[i + 1:i + degree + 1].mean() for i in range(n)], dtype=np.float64)


def _grid(gx, gy, gz):
    """Stack a tensor grid into (n1*n2*n3, 3) with x fastest."""
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    return np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)


def _insert_knot_1d(knots, ctrl, degree, u, axis):
    """Boehm knot insertion along one axis of a (n1, n2, n3, 3) net (input refinement)."""
    k = np.searchsorted(knots, u, side="right") - 1
    n = ctrl.shape[axis]
    new_shape = list(ctrl.shape)
    new_shape[axis] = n + 1
    out = np.empty(new_shape, dtype=np.float64)
    for i in range(n + 1):
        if i <= k - degree:
            a = 1.0
        elif i >= k + 1:
            a = 0.0
        else:
            a = (u - knots[i]) / (knots[i + degree] - knots[i])
        src_i = np.take(ctrl, min(i, n - 1), axis=axis)
        src_im1 = np.take(ctrl, max(i - 1, 0), axis=axis)
        idx = [slice(None)] * 4
        idx[axis] = i
        out[tuple(idx)] = a * src_i + (1.0 - a) * src_im1
    new_knots = np.insert(knots, k + 1, u)
    return new_knots, out


def macro_perturbed_cube(seed: int = 0, amp: float = 0.05, split: int = 2) -> MacroDesc:
    """Cubic Bezier cube with noisy control points, refined into split^3 tiles."""
    g = np.arange(4, dtype=np.float64) / 3.0
    ctrl = _grid(g, g, g)
    ctrl = ctrl + rng(seed).uniform(-amp, amp, size=ctrl.shape)
    net = ctrl.reshape(4, 4, 4, 3, order="F")  # net[i, j, k]
    knots = [np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.float64) for _ in range(3)]
    for axis in range(3):
        for s in range(1, split):
            knots[axis], net = _insert_knot_1d(knots[axis], net, 3, s / split, axis)
    n1, n2, n3 = net.shape[:3]
    ctrl = net.reshape(n1 * n2 * n3, 3, order="F")
    return MacroDesc(degree=(3, 3, 3), knots=tuple(knots), ctrl=np.ascontiguousarray(ctrl),
                     name=f"perturbed cube {split}x{split}x{split}")


def bezier_cube_reference(seed: int = 0, amp: float = 0.05) -> MacroDesc:
    """The unrefined noisy Bezier cube (used to check that refinement kept the geometry)."""
    g = np.arange(4, dtype=np.float64) / 3.0
    ctrl = _grid(g, g, g) + rng(seed).uniform(-amp, amp, size=(64, 3))
    knots = tuple(np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.float64) for _ in range(3))
    return MacroDesc(degree=(3, 3, 3), knots=knots, ctrl=ctrl, name="bezier cube")


def _uniform_net(nx, ny, nz, degree=3):
    knots = tuple(open_uniform_knots(n, degree) for n in (nx, ny, nz))
    gx, gy, gz = (greville(k, degree) for k in knots)
    return knots, _grid(gx, gy, gz)


def macro_affine_box(nx, ny, nz, lo=(0.0, 0.0, 0.0), size=None, degree=3) -> MacroDesc:
    """Affine map of [0,1]^3 onto a box (exact with a Greville net)."""
    size = size if size is not None else (float(nx), float(ny), float(nz))
    knots, g = _uniform_net(nx, ny, nz, degree)
    ctrl = np.asarray(lo, np.float64)[None, :] + g * np.asarray(size, np.float64)[None, :]
    return MacroDesc(degree=(degree,) * 3, knots=knots, ctrl=ctrl, name=f"box {nx}x{ny}x{nz}")


def macro_twisted_beam(nx, ny, nz, twist=0.5 * math.pi) -> MacroDesc:
    knots, g = _uniform_net(nx, ny, nz)
    x = nx * g[:, 0]
    y = ny * (g[:, 1] - 0.5)
    z = nz * (g[:, 2] - 0.5)
    phi = twist * x / nx
    c, s = np.cos(phi), np.sin(phi)
    ctrl = np.stack([x, c * y - s * z, s * y + c * z], axis=1)
    return MacroDesc(degree=(3, 3, 3), knots=knots, ctrl=ctrl, name=f"twisted beam {nx}x{ny}x{nz}")


def macro_quarter_arc(nx=20, ny=10, nz=10) -> MacroDesc:
    knots, g = _uniform_net(nx, ny, nz)
    x, y, z = nx * g[:, 0], ny * g[:, 1], nz * g[:, 2]
    phi = 0.5 * math.pi * x / nx
    rc = 2.0 * nx / math.pi
    r = rc + (y - 0.5 * ny)
    ctrl = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return MacroDesc(degree=(3, 3, 3), knots=knots, ctrl=ctrl, name=f"quarter arc {nx}x{ny}x{nz}")


def macro_cantilever(nx=20, ny=20, nz=5) -> MacroDesc:
    m = macro_affine_box(nx, ny, nz)
    m.name = f"cantilever plate {nx}x{ny}x{nz}"
    return m


def width_field(n_elem, seed: int = 0, mean=0.275, amp=0.125) -> np.ndarray:
    """Smooth sinusoidal strut-width field at tile centres, tile order ix + nx(iy + ny iz)."""
    nx, ny, nz = n_elem
    ph = rng(seed).uniform(0.0, 2.0 * math.pi, size=3)
    cx = (np.arange(nx) + 0.5) / nx
    cy = (np.arange(ny) + 0.5) / ny
    cz = (np.arange(nz) + 0.5) / nz
    X, Y, Z = np.meshgrid(cx, cy, cz, indexing="ij")
    w = mean + amp * np.sin(2 * math.pi * X + ph[0]) * np.sin(2 * math.pi * Y + ph[1]) \
        * np.sin(2 * math.pi * Z + ph[2])
    return np.ascontiguousarray(w.ravel(order="F"))


@dataclass
class Workload:
    name: str
    macro: MacroDesc
    n_e: int
    q: int
    width: float = 0.3
    widths: np.ndarray | None = None
    precisions: tuple = ("f64",)
    extra: dict = field(default_factory=dict)


def workload(name: str) -> Workload:
    """The five named workloads (shapes of the paper's lattices, synthetic)."""
    if name == "cube8":
        return Workload(name, macro_perturbed_cube(seed=0), n_e=2, q=2, precisions=("f64",))
    if name == "beam1000":
        return Workload(name, macro_twisted_beam(10, 10, 10), n_e=3, q=3, precisions=("f64", "f32"))
    if name == "beam125":      # small profiling case of the same shape (inputs still larger than L2)
        return Workload(name, macro_twisted_beam(5, 5, 5), n_e=3, q=3, precisions=("f64", "f32"))
    if name == "beam4000":
        return Workload(name, macro_twisted_beam(40, 10, 10), n_e=3, q=3,
                        precisions=("split_f16", "split_bf16", "tf32"))
    if name == "arc2000":
        m = macro_quarter_arc(20, 10, 10)
        return Workload(name, m, n_e=3, q=3, widths=width_field(m.n_elem, seed=0), precisions=("f32",))
    if name == "cantilever2000":
        return Workload(name, macro_cantilever(20, 20, 5), n_e=2, q=3, precisions=("f32", "f64"))
    raise KeyError(name)


WORKLOADS = ("cube8", "beam1000", "beam4000", "arc2000", "cantilever2000")
