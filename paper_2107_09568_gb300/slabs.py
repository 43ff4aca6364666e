"""One macro mesh split across GPUs: the host side of the tile-range entry points.

The tile matrices of eq. 58 are independent per tile (Sec. 3.2.4), and the tile-major global
numbering makes the CSR rows owned by a contiguous tile range [t0, t1) one contiguous range of
rows and values.  Rank r takes one contiguous range of tiles and assembles the complete rows its
tiles own with msasm_assemble_range, recomputing the halo -- the tiles of the next layer above
the range, whose glued lower faces carry points the range owns -- so the assembly moves no data
between ranks.  The compliance gradient of Sec. 4.1.2 (eq. 69-73) is a sum over tiles: each rank
computes its range's part with msasm_assemble_grad_range and one all-reduce adds them.
"""
from __future__ import annotations


def slab_ranges(n_tiles: int, world: int):
    """Balanced contiguous tile ranges [(t0, t1)] of the linear tile order, one per rank."""
    if world < 1 or n_tiles < 0:
        raise ValueError("need world >= 1 and n_tiles >= 0")
    return [(n_tiles * r // world, n_tiles * (r + 1) // world) for r in range(world)]


def halo_end(t1: int, n_elem) -> int:
    """End of the tiles whose blocks reach the rows owned by a range ending at t1: a tile t is glued
    to t - 1, t - nx and t - nx ny through its lower faces, so the tiles up to one layer (nx ny)
    above the range are the last that add to its rows."""
    nx, ny, nz = (int(v) for v in n_elem)
    return min(nx * ny * nz, t1 + nx * ny)


def allreduce_gradient(grad, dist):
    """Sum the ranks' partial dL/dP (each from its tile range) in place: the whole gradient."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    return grad
