"""One mesh split across ranks, host side, on CPU: world size 2 over gloo.

Each rank takes its contiguous tile range from slabs.slab_ranges and the halo end from
slabs.halo_end (the same rule as msasm_plan_range), and -- with the oracle as the compute
engine -- checks that the range owns one contiguous block of point ids, that every tile holding
one of its points lies in [t0, halo_end), and that the blocks of those tiles alone give its rows
of the whole-mesh stiffness.  The gathered rows of all ranks are the whole matrix, and the
ranks' partial compliance gradients (eq. 69-73 summed over their own tiles), added by
slabs.allreduce_gradient, are the whole gradient."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import synth  # noqa: E402
from paper_2107_09568_gb300 import slabs  # noqa: E402


def _problem():
    from oracle.assembly import Problem
    return Problem(synth.micro_cross(2), synth.macro_twisted_beam(3, 2, 2), 1)


def _owner(prob):
    own = np.full(prob.n_points, prob.mmap.n_tiles, dtype=np.int64)
    for t in range(prob.mmap.n_tiles):
        own[prob.gmap[t]] = np.minimum(own[prob.gmap[t]], t)
    return own


def _check_range(prob, t0, t1):
    """(p0, p1, window of values) of the rows owned by tiles [t0, t1), from the blocks of [t0, halo_end)."""
    from oracle.assembly import nzdata_lookup, scatter_csr
    own = _owner(prob)
    ids = np.nonzero((own >= t0) & (own < t1))[0]
    p0, p1 = int((own < t0).sum()), int((own < t1).sum())
    assert np.array_equal(ids, np.arange(p0, p1))                  # one contiguous block of ids
    he = slabs.halo_end(t1, prob.mmap.n_elem)
    for g in ids:                                                  # every tile reaching the rows is computed
        tiles = np.nonzero((prob.gmap == g).any(axis=1))[0]
        assert tiles.min() >= t0 and tiles.max() < he, (g, tiles, t0, he)
    tiles = list(range(t0, he))
    nz = nzdata_lookup(prob.T, prob.mmap, prob.q, prob.lam, prob.mu, tiles=tiles) if tiles else []
    vals = scatter_csr(prob.tile, prob.gmap, prob.rowptr, prob.col, zip(tiles, nz))
    v0, v1 = int(prob.rowptr[3 * p0]), int(prob.rowptr[3 * p1])
    return p0, p1, vals[v0:v1]


def _partial_gradient(prob, u, coords, t0, t1, h=1e-30):
    """The part of d(u^T K u)/dP from tiles [t0, t1), by the oracle's complex step."""
    from oracle.adjoint import tile_quadratic, tiles_of_control_point
    out = []
    for k, p in coords:
        c = prob.mmap.macro.ctrl.astype(np.complex128).copy()
        c[k, p] += 1j * h
        q = sum(tile_quadratic(prob, t, u.reshape(-1, 3), c) for t in tiles_of_control_point(prob, k)
                if t0 <= t < t1)
        out.append(np.imag(q) / h)
    return np.array(out)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        t0, t1 = slabs.slab_ranges(prob.mmap.n_tiles, world)[rank]
        p0, p1, window = _check_range(prob, t0, t1)
        rows = [None] * world
        dist.all_gather_object(rows, (p0, p1, window))
        rng = np.random.default_rng(11)
        u = rng.normal(size=3 * prob.n_points)
        coords = [(int(k), int(p)) for k, p in zip(rng.choice(prob.mmap.macro.ctrl.shape[0], 6, replace=False),
                                                   rng.integers(0, 3, 6))]
        g = torch.tensor(_partial_gradient(prob, u, coords, t0, t1))
        slabs.allreduce_gradient(g, dist)
        out[rank] = (rows, g.numpy(), u, coords)
    finally:
        dist.destroy_process_group()


def test_slab_partition_halo_and_gradient_allreduce_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    from oracle.adjoint import gradient_complex_step
    prob = _problem()
    whole = prob.assemble_lookup()
    for r in range(world):
        rows, g, u, coords = out[r]
        assert rows[0][0] == 0 and rows[-1][1] == prob.n_points
        assert all(rows[i][1] == rows[i + 1][0] for i in range(world - 1))   # the ranges tile the points
        got = np.concatenate([w for _, _, w in rows])
        assert got.shape == whole.shape
        assert np.linalg.norm(got - whole) <= 1e-14 * np.linalg.norm(whole)
        ref = gradient_complex_step(prob, u, coords)
        assert np.allclose(g, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("world", [1, 3, 5])
def test_slab_ranges_cover_every_tile_once(world):
    """Uneven partitions (a range may end mid-layer) still own contiguous ids and reach only [t0, halo_end)."""
    prob = _problem()
    rng_list = slabs.slab_ranges(prob.mmap.n_tiles, world)
    assert rng_list[0][0] == 0 and rng_list[-1][1] == prob.mmap.n_tiles
    assert all(a[1] == b[0] for a, b in zip(rng_list, rng_list[1:]))
    whole = prob.assemble_lookup()
    parts = [_check_range(prob, t0, t1)[2] for t0, t1 in rng_list]
    got = np.concatenate(parts)
    assert np.linalg.norm(got - whole) <= 1e-14 * np.linalg.norm(whole)
