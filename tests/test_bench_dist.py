"""Host logic of bench.py: the max-over-ranks timing and the whole-job rate with world size 2 over
gloo on CPU (the path every N > 1 run takes, with NCCL there), and the clock-sample window."""
import os
import socket
import time

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                        # rank 1 is the slow one
        total = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.whole_job_rate(1000, world, 3, total)
        dist.barrier()
        out[rank] = (total, value)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        total, value = out[r]
        assert total == 15.0                          # every rank sees the slowest rank's time
        assert value == pytest.approx(1000 * 2 * 3 / 0.015)


def test_single_process_is_identity():
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.whole_job_rate(1000, 1, 10, 100.0) == pytest.approx(1e5)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_samples_are_those_of_the_timed_region(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clk.csv")
    c.proc, c.f = _FakeProc(), open(os.devnull, "w")
    t0 = time.time()
    c.t_begin, c.t_end = t0 + 1.0, t0 + 2.0

    def line(t, mhz, power_cap="Not Active"):
        stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)
        return f"{stamp}, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {power_cap}\n"

    with open(c.path, "w") as f:
        f.write(line(t0 + 0.2, 345))                  # idle, before the region
        f.write(line(t0 + 1.3, 2070))
        f.write(line(t0 + 1.6, 2055, "Active"))
        f.write(line(t0 + 2.8, 900))                  # after the region
    r = c.stop()
    assert r["samples"] == 2 and r["samples_total"] == 4 and r["window"] == "timed region"
    assert r["sm_mhz"] == pytest.approx((2070 + 2055) / 2)
    assert r["reasons"] == ["sw_power_cap"]


def test_cpulist_parsing_and_binding_fallback():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("") == set()
    before = os.sched_getaffinity(0)
    r = bench.bind_to_gpu_local_cpus(0)           # no GPU here: nothing is changed
    assert r["bound"] is False and os.sched_getaffinity(0) == before


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_slab_setup_of_the_multi_gpu_bench(world):
    """bench.py --gpus N: every rank gets the same per-GPU work (the 4000 tiles of the 40x10x10 beam,
    weak scaling along z), the ranks' slabs tile the grown mesh, and each recomputes at most one layer."""
    ranges = [bench.slab_setup("beam4000", world, r) for r in range(world)]
    macro, n_elem, n_total, _, _, _ = ranges[0]
    assert n_elem == (40, 10, 10 * world) and n_total == 4000 * world
    assert macro.ctrl.shape[0] == 43 * 13 * (10 * world + 3)      # degree-3 net of the grown beam
    assert ranges[0][3] == 0 and ranges[-1][4] == n_total
    for r, (_, _, _, t0, t1, he) in enumerate(ranges):
        assert t1 - t0 == 4000                                     # the same work on every GPU
        if r + 1 < world:
            assert ranges[r + 1][3] == t1                          # consecutive slabs
            assert he == t1 + 400                                  # one 40 x 10 layer of halo
        else:
            assert he == n_total


def test_traffic_figure_follows_the_kernel_code_not_its_comments():
    """The DRAM traffic in the bench line is tied to a digest of the contraction's code: a comment
    edit keeps it, a code edit makes the line report traffic as null."""
    base = "int a = 1;  // one\n/* block\n comment */\nint b = a;\n"
    assert bench._code_only(base) == bench._code_only(base.replace("// one", "// two").replace("block", "x"))
    assert bench._code_only(base) != bench._code_only(base.replace("int b = a;", "int b = a + 1;"))
    d = bench.kernel_source_digest("contract_emu_kernel")
    assert (("contract_emu_kernel", "beam4000", "f64_emu") in bench.NCU_TRAFFIC
            and bench.NCU_TRAFFIC[("contract_emu_kernel", "beam4000", "f64_emu")][2] == d)
