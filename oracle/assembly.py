"""Global numbering, CSR structure and the two assembly forms (Sec. 3.2.4 and 3.3).

Conventions (readings where the paper leaves a choice):
* DOF of component alpha of global point g is row 3 g + alpha.
* A control point on the xi_d = 0 face of tile t with a neighbour t - e_d is the
  same point as the matching point on the xi_d = 1 face of t - e_d.  Its owner is
  the tile with the lowest linear index holding it; global ids are assigned in
  order (owner tile, local id).
* CSR: row pointer int64, column index int32 ascending, full symmetric storage.
  The stored pattern is the union over tiles of all ordered pairs of eq. 56.
* Tile block (eq. 49): K[(A,alpha),(B,beta)] = sum_ij int phi_A,i phi_B,j A_ij[alpha,beta];
  the block (B, A) is its transpose.
"""
from __future__ import annotations

import numpy as np

from . import pullback, quadrature
from .macro import MacroMap


# ------------------------------------------------------------------ numbering / structure
def numbering(tile, mmap: MacroMap):
    """gmap[t, A] -> global point id; returns (gmap (m_M, n_T) int64, n_points)."""
    nx, ny, nz = mmap.n_elem
    m = mmap.n_tiles
    gmap = -np.ones((m, tile.n_T), dtype=np.int64)
    nxt = 0
    strides = (1, nx, nx * ny)
    for t in range(m):
        idx = mmap.tile_index(t)
        shared = {}
        for d in range(3):
            if idx[d] > 0:
                lower_face = tile.faces[2 * d]        # xi_d = 0 of tile t
                upper_face = tile.faces[2 * d + 1]    # xi_d = 1 of tile t - e_d
                for pos, A in enumerate(lower_face):
                    shared[int(A)] = gmap[t - strides[d], upper_face[pos]]
        for A in range(tile.n_T):
            if A in shared:
                gmap[t, A] = shared[A]
            else:
                gmap[t, A] = nxt
                nxt += 1
    return gmap, nxt


def ordered_local_pairs(tile):
    """All ordered (A, B) with overlapping supports, A == B included."""
    P = tile.pairs
    off = P[P[:, 0] != P[:, 1]]
    return np.concatenate([P, off[:, ::-1]], axis=0)


def point_adjacency(tile, gmap, n_points):
    """Point-level pattern: (pptr int64 (n_points+1), pcol int64) sorted unique per row."""
    op = ordered_local_pairs(tile)
    keys = []
    for t in range(gmap.shape[0]):
        g = gmap[t]
        keys.append(g[op[:, 0]] * n_points + g[op[:, 1]])
    keys = np.unique(np.concatenate(keys))
    rows = keys // n_points
    pcol = keys % n_points
    pptr = np.zeros(n_points + 1, dtype=np.int64)
    np.add.at(pptr, rows + 1, 1)
    return np.cumsum(pptr), pcol


def csr_structure(pptr, pcol):
    """Expand the point pattern to the 3x3-block DOF pattern (rowptr int64, col int32)."""
    n_points = len(pptr) - 1
    deg = np.diff(pptr)
    rowlen = np.repeat(3 * deg, 3)
    rowptr = np.zeros(3 * n_points + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(rowlen)
    col = np.empty(rowptr[-1], dtype=np.int64)
    for g in range(n_points):
        cols = (3 * pcol[pptr[g]:pptr[g + 1]][:, None] + np.arange(3)[None, :]).ravel()
        for a in range(3):
            col[rowptr[3 * g + a]:rowptr[3 * g + a + 1]] = cols
    return rowptr, col.astype(np.int32)


# ------------------------------------------------------------------ lookup ("pi") form
def node_jacobians(mmap: MacroMap, t: int, q: int, ctrl=None):
    """J^(t) at the (q+1)^3 interpolation nodes, shape (n_pi, 3, 3)."""
    _, J = mmap.tile_map(t, quadrature.tensor_nodes(q), ctrl)
    return J


def coefficient_block(mmap, t, q, lam, mu, ctrl=None):
    """mat[<A>] columns of tile t: (9 n_pi, 9), row (C, i, j), column (alpha, beta) (eq. 42, 58)."""
    A = pullback.macro_field(node_jacobians(mmap, t, q, ctrl), lam, mu)   # (n_pi, i, j, a, b)
    n_pi = A.shape[0]
    return A.reshape(n_pi * 9, 9)


def tile_blocks_lookup(T, mmap, t, q, lam, mu, ctrl=None):
    """nzdata of one tile, eq. 58: (n_nz, 3, 3) = mat[K] (n_nz, 9 n_pi) . mat[<A>] (9 n_pi, 9)."""
    n_nz = T.shape[0]
    return (T.reshape(n_nz, -1) @ coefficient_block(mmap, t, q, lam, mu, ctrl)).reshape(n_nz, 3, 3)


def nzdata_lookup(T, mmap, q, lam, mu, ctrl=None, tiles=None):
    """All tile blocks as one matrix product, eq. 58: returns (n_tiles, n_nz, 3, 3)."""
    tiles = range(mmap.n_tiles) if tiles is None else tiles
    B = np.concatenate([coefficient_block(mmap, t, q, lam, mu, ctrl) for t in tiles], axis=1)
    n_nz = T.shape[0]
    C = T.reshape(n_nz, -1) @ B                                   # (n_nz, 9 m)
    return C.reshape(n_nz, len(tiles), 3, 3).transpose(1, 0, 2, 3)


# ------------------------------------------------------------------ standard ("bullet") form
def tile_blocks_quadrature(tile, mmap, t, lam, mu, n_g=6, ctrl=None):
    """Tile blocks (n_nz, 3, 3) by full Gauss quadrature on the composed map (Sec. 3.3, ref. 36).

    On each micro element, theta -> xi = T^r(theta) -> x = M^(t)(xi); physical gradients
    grad_x phi = J_M^-T J_T^-T grad_theta R, weight w |det J_T| |det J_M|, and the isotropic
    integrand lam d_a phi_A d_b phi_B + mu (grad phi_A . grad phi_B delta_ab + d_b phi_A d_a phi_B).
    """
    K = np.zeros((tile.n_nz, 3, 3))
    g1, w1 = quadrature.gauss_legendre(n_g)
    eye = np.eye(3)
    for el in tile.elements:
        P = tile.patches[el["patch"]]
        lo, hi = P["lo"], P["hi"]
        pts = [el["th_lo"][d] + (el["th_hi"][d] - el["th_lo"][d]) * g1 for d in range(3)]
        wts = [(el["th_hi"][d] - el["th_lo"][d]) * w1 for d in range(3)]
        theta = np.array([(a, b, c) for c in pts[2] for b in pts[1] for a in pts[0]])
        wgt = np.array([wa * wb * wc for wc in wts[2] for wb in wts[1] for wa in wts[0]])
        xi = lo + (hi - lo) * theta
        _, JM = mmap.tile_map(t, xi, ctrl)                         # (g, 3, 3)
        detM = np.abs(np.linalg.det(JM))
        w = wgt * np.prod(hi - lo) * detM
        _, grads = tile.patch_basis(el["patch"], theta)
        nf = P["nfun"]
        cols = [a1 + nf[0] * (a2 + nf[1] * a3) for (a1, a2, a3) in el["loc"]]
        dxi = grads[:, cols, :] / (hi - lo)                        # (g, 27, 3) d/dxi
        dx = np.einsum("gip,gai->gap", np.linalg.inv(JM), dxi)     # J_M^-T grad_xi
        dot = np.einsum("gap,gbp->gab", dx, dx)
        Kl = (lam * np.einsum("g,gaq,gbr->aqbr", w, dx, dx)
              + mu * np.einsum("g,gab,qr->aqbr", w, dot, eye)
              + mu * np.einsum("g,gar,gbq->aqbr", w, dx, dx))
        ids = el["ids"]
        for a, A in enumerate(ids):
            for b, B in enumerate(ids):
                if A <= B:
                    K[tile.pair_index[(A, B)]] += Kl[a, :, b, :]
    return K


# ------------------------------------------------------------------ sparse assembly (step 4)
def scatter_csr(tile, gmap, rowptr, col, blocks_by_tile):
    """Add every tile block and its transpose into CSR values aligned with (rowptr, col)."""
    n_rows = len(rowptr) - 1
    row_of = np.repeat(np.arange(n_rows, dtype=np.int64), np.diff(rowptr))
    struct_keys = row_of * (n_rows + 1) + col.astype(np.int64)
    P = tile.pairs
    rows_l, cols_l, vals_l = [], [], []
    ab = np.arange(3)
    for t, Kt in blocks_by_tile:
        gA, gB = gmap[t, P[:, 0]], gmap[t, P[:, 1]]
        shp = (len(P), 3, 3)
        r = np.broadcast_to(3 * gA[:, None, None] + ab[None, :, None], shp)
        c = np.broadcast_to(3 * gB[:, None, None] + ab[None, None, :], shp)
        rows_l.append(r.ravel()); cols_l.append(c.ravel()); vals_l.append(Kt.ravel())
        off = P[:, 0] != P[:, 1]
        # transpose block: entry (3 gB + beta, 3 gA + alpha) = K[m, alpha, beta]
        shp = (int(off.sum()), 3, 3)
        rT = np.broadcast_to(3 * gB[off][:, None, None] + ab[None, None, :], shp)
        cT = np.broadcast_to(3 * gA[off][:, None, None] + ab[None, :, None], shp)
        rows_l.append(rT.ravel()); cols_l.append(cT.ravel()); vals_l.append(Kt[off].ravel())
    rows = np.concatenate(rows_l); cols = np.concatenate(cols_l); vals = np.concatenate(vals_l)
    pos = np.searchsorted(struct_keys, rows * (n_rows + 1) + cols)
    assert np.all(struct_keys[pos] == rows * (n_rows + 1) + cols), "entry outside the pattern"
    return np.bincount(pos, weights=vals, minlength=len(col))


class Problem:
    """Everything the oracle needs for one workload: tile, macro map, numbering, table."""

    def __init__(self, micro, macro, q, E=1.0, nu=0.3, table=None, structure=True):
        from .micro import ReferenceTile
        from . import tables
        self.tile = ReferenceTile(micro)
        self.mmap = MacroMap(macro)
        self.q = q
        self.lam, self.mu = pullback.lame(E, nu)
        self.gmap, self.n_points = numbering(self.tile, self.mmap)
        self.T = tables.build_table(self.tile, q) if table is None else table
        if structure:
            self.pptr, self.pcol = point_adjacency(self.tile, self.gmap, self.n_points)
            self.rowptr, self.col = csr_structure(self.pptr, self.pcol)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def assemble_lookup(self, ctrl=None):
        nz = nzdata_lookup(self.T, self.mmap, self.q, self.lam, self.mu, ctrl)
        return scatter_csr(self.tile, self.gmap, self.rowptr, self.col, enumerate(nz))

    def assemble_quadrature(self, n_g=6, ctrl=None):
        blocks = ((t, tile_blocks_quadrature(self.tile, self.mmap, t, self.lam, self.mu, n_g, ctrl))
                  for t in range(self.mmap.n_tiles))
        return scatter_csr(self.tile, self.gmap, self.rowptr, self.col, blocks)

    def point_positions(self, ctrl=None):
        """Physical position M^(t)(t_A) of every global control point (for rigid modes)."""
        X = np.zeros((self.n_points, 3))
        for t in range(self.mmap.n_tiles):
            x, _ = self.mmap.tile_map(t, self.tile.points, ctrl)
            X[self.gmap[t]] = x
        return X


def point_rows(prob: "Problem", points, ctrl=None, blocks_fn=None):
    """CSR rows of sampled global points without forming K: {g: (neighbour ids, (deg, 3, 3) blocks)}.

    Row block (g, h) = sum over tiles tau holding g of K_tau[(A, B)] (A = local g, B = local h),
    using the stored upper block or the transpose of (B, A).  ``blocks_fn(t)`` returns the
    (n_nz, 3, 3) tile blocks (default: the lookup form, eq. 58).
    """
    tile = prob.tile
    if blocks_fn is None:
        blocks_fn = lambda t: tile_blocks_lookup(prob.T, prob.mmap, t, prob.q, prob.lam, prob.mu, ctrl)
    cache = {}
    out = {}
    P = tile.pairs
    for g in points:
        acc = {}
        for t, A in np.argwhere(prob.gmap == g):
            if t not in cache:
                cache[t] = blocks_fn(int(t))
            Kt = cache[t]
            up = np.nonzero(P[:, 0] == A)[0]
            lo = np.nonzero((P[:, 1] == A) & (P[:, 0] != A))[0]
            for m in up:
                h = int(prob.gmap[t, P[m, 1]])
                acc[h] = acc.get(h, 0.0) + Kt[m]
            for m in lo:
                h = int(prob.gmap[t, P[m, 0]])
                acc[h] = acc.get(h, 0.0) + Kt[m].T
        hs = np.array(sorted(acc), dtype=np.int64)
        out[int(g)] = (hs, np.array([acc[h] for h in hs]))
    return out
