"""Throughput of the multiscale lookup-table stiffness assembly on one GB300.

One step = one full assembly of the workload's global CSR stiffness through the
C ABI: pullback + interpolation of the macro field (step 1), the table contraction
(step 3, eq. 58) and the CSR scatter (step 4), all tiles, inputs resident in HBM.

Default workload: the 40x10x10 twisted beam (4000 tiles, cross cell with 3x3x3
elements per patch, q = 3), the largest of the five lattice workloads that one GPU
holds, in its FP64-accurate form: the contraction emulates FP64 exactly with BF16
tensor-core slices (within 1e-12 of the FP64 CUDA-core form).  The same JSON line
carries every other precision form on that workload, the learned surrogate on the
graded quarter arc (2000 tiles) and the adjoint gradient on the cantilever plate
(2000 tiles), each against the plain FP64 GPU form.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision f64_emu|f64|f32|...] [--workload beam4000|...]

--impl reference times the FP64 CPU oracle (the only baseline there is: the
paper's code is not available) on a bounded sample of tiles per step.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tiles/s and stiffness GB/s vs FP64 GPU lookup form at stated rel. error"
WORKLOAD_TEXT = {
    "beam1000": "twisted beam 10x10x10 tiles (90-degree twist), cross cell 7 patches x 3^3 degree-2 elements, "
                "q=3 (64 nodes), E=1 nu=0.3",
    "cube8": "perturbed cubic cube split 2x2x2, cross cell 7 patches x 2^3 elements, q=2",
    "beam125": "twisted beam 5x5x5 tiles, cross cell n_e=3, q=3 (profiling case)",
    "beam4000": "twisted beam 40x10x10 tiles (90-degree twist), cross cell 7 patches x 3^3 degree-2 elements, "
                "q=3 (64 nodes), E=1 nu=0.3",
    "cantilever2000": "cantilever plate 20x20x5 tiles, cross cell n_e=2, q=3",
    "arc2000": "quarter arc 20x10x10 tiles, cross cell n_e=3, q=3 (uniform width 0.3)",
}
L2_POLICY = "256 MB buffer written between timed steps (L2 is 129 MB); each step also writes the CSR values"
FORMS = "f64,f32,split_f16,split_bf16,tf32,tf32x3,f64_emu"


def slab_setup(workload, world, rank):
    """The mesh and this rank's tiles: the workload itself at one GPU; with N > 1 GPUs (weak scaling)
    the same twisted beam with N times as many layers along z, rank r taking one contiguous slab of the
    tiles and recomputing the layer above it.  Returns (macro, mesh, tiles, t0, t1, halo end)."""
    import synth
    from paper_2107_09568_gb300 import slabs
    w = synth.workload(workload)
    macro = w.macro
    if world > 1:
        if not workload.startswith("beam"):
            raise SystemExit("--gpus N > 1 splits a twisted-beam workload (beam125, beam1000, beam4000)")
        nx, ny, nz = (int(v) for v in w.macro.n_elem)
        macro = synth.macro_twisted_beam(nx, ny, nz * world)
    n_elem = tuple(int(v) for v in macro.n_elem)
    n_total = n_elem[0] * n_elem[1] * n_elem[2]
    t0, t1 = slabs.slab_ranges(n_total, world)[rank]
    return macro, n_elem, n_total, t0, t1, slabs.halo_end(t1, n_elem)


def workload_config(name):
    """The `config` object of the JSON line: the workload alone, identical in both arms."""
    import synth
    w = synth.workload(name)
    n = tuple(int(x) for x in w.macro.n_elem)
    return {"workload": name, "text": WORKLOAD_TEXT.get(name, ""), "tiles": n[0] * n[1] * n[2],
            "mesh": list(n), "micro_elements_per_patch_dir": w.n_e, "q": w.q, "l2": L2_POLICY}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64_emu")
    ap.add_argument("--workload", default="beam4000")
    ap.add_argument("--forms", default=FORMS, help="comma list of precision forms to report beside the headline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the surrogate and adjoint workloads")
    ap.add_argument("--report", default="", help="comma list of: forms1000, forms4000, surrogate, adjoint, volume, linop, projection, cpu_forms "
                                                 "(prints a JSON report instead of the bench line)")
    return ap.parse_args()


def parse_cpulist(text):
    """'0-3,8,10-11' -> {0, 1, 2, 3, 8, 10, 11}."""
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.update(range(int(a), int(b or a) + 1))
    return cpus


def bind_to_gpu_local_cpus(gpu):
    """Restrict this process to the host CPUs local to GPU `gpu` (its PCI device's local_cpulist),
    so that pinned host buffers allocated afterwards sit in the host memory next to that GPU (a
    far NUMA node cuts the device-to-host rate).  Returns a description of what was done."""
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={gpu}", "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        dev = f"{int(dom, 16):04x}:{rest.lower()}"
        with open(f"/sys/bus/pci/devices/{dev}/local_cpulist") as f:
            local = parse_cpulist(f.read())
        avail = os.sched_getaffinity(0)
        use = local & avail
        if not use or use == avail:
            return {"pci": dev, "cpus": len(avail), "bound": False}
        os.sched_setaffinity(0, use)
        return {"pci": dev, "cpus": len(use), "of": len(avail), "bound": True}
    except Exception as e:                       # no nvidia-smi, no sysfs entry: leave it as it is
        return {"bound": False, "why": type(e).__name__}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons; only the samples taken inside the
    timed region (mark_begin .. mark_end, host wall clock) are kept."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=40):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.path = os.path.join("/tmp", f"msasm_clocks_{os.getpid()}.csv")
        self.t_begin = self.t_end = None

    def mark_begin(self):
        self.t_begin = time.time()

    def mark_end(self):
        self.t_end = time.time()

    def wait_first_sample(self, timeout=3.0):
        """Block until nvidia-smi has written a line (it takes a moment to start)."""
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < timeout:
            if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        n_all, kept, other = 0, [], []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            n_all += 1
            try:
                whole, frac = (parts[0].split(".") + ["0"])[:2]
                ts = time.mktime(time.strptime(whole, "%Y/%m/%d %H:%M:%S")) + float("0." + frac)
            except (ValueError, IndexError):
                ts = None
            try:
                rec = (float(parts[1]), float(parts[2]), parts[5:9])
            except ValueError:
                continue
            inside = ts is not None and self.t_begin is not None and self.t_begin - 0.05 <= ts <= self.t_end + 0.05
            (kept if inside else other).append(rec)
        window = "timed region"
        if not kept:                       # no sample inside a very short region: report the nearest ones
            kept, window = other[-2:], "just before and after the timed region"
        for f_sm, f_max, flags in kept:
            sm.append(f_sm); smax.append(f_max)
            for n, v in zip(names, flags):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "samples_total": n_all, "window": window, "reasons": sorted(reasons)}


def max_over_ranks(x, dist, device="cpu"):
    """The largest of every rank's x (the job ends when its slowest rank does)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, steps, max_ms):
    """Units all ranks processed per second of the slowest rank (weak scaling: fixed units per rank)."""
    return units_per_rank * world * steps / (max_ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 CUDA-core peak: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (GB300 FP64 is 1/64 of B200's per SM)
FP64_ALU_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); the profile named beside each figure gives the
# command.  Keyed by (kernel, workload, precision); the last field is the digest of the kernel's
# source files when the counters were taken: when the source has changed since, the figure no
# longer describes the kernel and the line reports traffic as null.
NCU_TRAFFIC = {
    ("contract_emu_kernel", "beam4000", "f64_emu"): (4209443584 + 6766186752, "profiles/contract_emu_beam4000.md",
                                                     "96322d7eb7c2b88f"),
}
KERNEL_SOURCES = {
    "contract_emu_kernel": ("contract_emu.cu", "tc_ptx.cuh"),
    "contract_tc_kernel": ("contract_tc.cu", "tc_ptx.cuh"),
    "scatter": ("scatter.cu",),
}


def _code_only(text):
    """C/C++/CUDA source without comments, blank lines or trailing blanks (a comment edit does not
    change the compiled kernel, so it does not make counters taken before it stale)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_digest(kernel):
    """sha256 (first 16 hex digits) of the code (comments stripped) of the files a kernel is compiled from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2107_09568_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def contraction_flops(n_nz, n_pi, n_tiles):
    return 2.0 * n_nz * 9 * n_pi * 9 * n_tiles


# tensor-core products issued per algorithmic product, and the unit's peak relative to BF16 dense
TC_PRODUCTS = {"split_f16": 3, "split_bf16": 3, "tf32": 1, "tf32x3": 3, "f64_emu": 28, "f32": 10}
TC_PEAK_RATIO = {"split_f16": 1.0, "split_bf16": 1.0, "tf32": 1.1 / 2.25, "tf32x3": 1.1 / 2.25, "f64_emu": 1.0,
                 "f32": 1.0}


def oracle_problem(workload):
    """The oracle's lookup-form problem of a workload (tables and numbering; set-up, not timed)."""
    import synth
    from oracle.assembly import Problem
    w = synth.workload(workload)
    return Problem(synth.micro_cross(w.n_e, w.width), w.macro, w.q, structure=False)


def cpu_reference_time(prob, n_sample, seed=0):
    """FP64 oracle (lookup form: pullback, contraction, scatter) on a sample of tiles; returns (s, tiles)."""
    from oracle.assembly import nzdata_lookup
    rng = np.random.default_rng(seed)
    tiles = np.sort(rng.choice(prob.mmap.n_tiles, min(n_sample, prob.mmap.n_tiles), replace=False))
    t0 = time.perf_counter()
    nz = nzdata_lookup(prob.T, prob.mmap, prob.q, prob.lam, prob.mu, tiles=list(tiles))
    # step 4 for the sample: the values land in a COO stream with global (row, col) of every entry
    P = prob.tile.pairs
    total = 0.0
    for k, t in enumerate(tiles):
        g = prob.gmap[t]
        rows = 3 * g[P[:, 0]][:, None, None] + np.arange(3)[None, :, None]
        cols = 3 * g[P[:, 1]][:, None, None] + np.arange(3)[None, None, :]
        keys = np.broadcast_to(rows * 10 ** 9 + cols, nz[k].shape)
        order = np.argsort(keys, axis=None)
        total += float(np.take(nz[k].ravel(), order).sum())
    dt = time.perf_counter() - t0
    return dt, len(tiles)


def cpu_forms_report(workload, n_tiles=2):
    """The oracle's lookup form against its full-quadrature (standard) form on the host cores, per tile
    (the paper's T_cost of eq. 64, here for the FP64 CPU oracle): context only."""
    import synth
    from oracle.assembly import Problem, nzdata_lookup, tile_blocks_quadrature
    w = synth.workload(workload)
    prob = Problem(synth.micro_cross(w.n_e), w.macro, w.q, structure=False)
    tiles = list(range(n_tiles))
    t0 = time.perf_counter()
    nzdata_lookup(prob.T, prob.mmap, prob.q, prob.lam, prob.mu, tiles=tiles)
    t_look = (time.perf_counter() - t0) / n_tiles
    t0 = time.perf_counter()
    for t in tiles:
        tile_blocks_quadrature(prob.tile, prob.mmap, t, prob.lam, prob.mu)
    t_quad = (time.perf_counter() - t0) / n_tiles
    return {"tiles": n_tiles, "lookup_s_per_tile": t_look, "quadrature_s_per_tile": t_quad,
            "t_cost": t_quad / t_look, "cores": threads_used()}


def threads_used():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, a bounded sample of the workload's tiles
    per step.  Under torchrun only rank 0 runs it; the other ranks exit at once."""
    if rank != 0:
        return 0
    prob = oracle_problem(args.workload)
    per_step = 16 if args.workload in ("beam1000", "beam4000", "arc2000") else 8
    for k in range(args.warmup):
        cpu_reference_time(prob, max(2, per_step // 4), seed=1000 + k)
    times, tiles = [], 0
    for k in range(args.steps):
        dt, n = cpu_reference_time(prob, per_step, seed=k)
        times.append(dt)
        tiles += n
    total = sum(times)
    value = tiles / total
    cores = threads_used()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload),
            "execution": "FP64 oracle on the host cores (numpy/BLAS), rank 0 only",
            "cpu_baseline": {"value": value, "unit": "tiles/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random tiles per step, FP64 lookup form "
                                       "(pullback, contraction, per-tile scatter ordering)"},
            "e2e": {"value": value, "unit": "tiles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_report(args):
    import torch
    import paper_2107_09568_gb300 as msasm
    from paper_2107_09568_gb300 import workloads as wl
    msasm.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    forms = ["f64_emu", "f32", "split_f16", "split_bf16", "tf32", "tf32x3"]
    out = {}
    for item in args.report.split(","):
        t0 = time.perf_counter()
        if item == "forms1000":
            out[item] = wl.precision_forms("beam1000", forms, flush)
        elif item == "forms4000":
            out[item] = wl.precision_forms("beam4000", forms, flush)
        elif item == "surrogate":
            out[item] = wl.surrogate(flush)
        elif item == "adjoint":
            out[item] = wl.adjoint(flush)
        elif item == "volume":
            out[item] = wl.volume(flush)
        elif item == "linop":
            out[item] = wl.linop(flush, args.workload if args.workload != "beam4000" else "beam1000")
        elif item == "projection":
            out[item] = wl.projection(flush)
        elif item == "cpu_forms":
            out[item] = cpu_forms_report(args.workload)
        else:
            continue
        out[item]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def roofline_of(stage_avg, prec, tab, n_tiles, nnz, pk, pk_kind, workload):
    """The dominant kernel's algorithmic rate against its peak (a measured one where there is one)."""
    names = ["pullback", "contraction", "scatter"]
    dom = int(np.argmax(stage_avg))
    vbytes = 8 if prec in ("f64", "f64_emu") else 4
    K = 9 * tab.n_pi
    flops = contraction_flops(tab.n_nz, tab.n_pi, n_tiles)
    nz_bytes = 9 * n_tiles * tab.n_nz * vbytes
    scatter_bytes = nz_bytes + nnz * vbytes                  # nzdata read, values written (once each)
    pull_bytes = 9 * n_tiles * K * 8
    if names[dom] == "contraction" and prec == "f64":
        alu_peak = FP64_ALU_PEAK_TFLOPS
        ach = flops / (stage_avg[1] / 1e3) / 1e12
        roof = {"kernel": f"contract_simt_{prec}", "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": None,
                "peak_source": "derived: 152 SMs x lanes per SM x 2 flop x 2.07 GHz",
                "algorithmic": f"2*n_nz*9n_pi*9m = {flops:.4g} flop per launch"}
    elif names[dom] == "contraction":
        # the form's own peak: the tensor pipe's measured burst rate (the kernel is timed in steps of
        # tens of ms) divided by the products one multiply-add of the emulated type costs (28 BF16
        # products per FP64-accurate one, 3 per split-FP32 one, 1 for TF32)
        n_prod = TC_PRODUCTS.get(prec, 1)
        ratio = TC_PEAK_RATIO.get(prec, 1.0)
        peak = pk["bf16_tflops"] * ratio / n_prod
        peak_sus = pk["bf16_tflops_sustained"] * ratio / n_prod
        ach = flops / (stage_avg[1] / 1e3) / 1e12
        roof = {"kernel": "contract_emu_kernel" if prec in ("f64_emu", "f32") else "contract_tc_kernel", "bound": "tensor",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": f"{pk_kind} bf16 burst {pk['bf16_tflops']}"
                               + (" x 1.1/2.25 (tf32 nominal ratio)" if "tf32" in prec else "")
                               + f" / {n_prod} products per {prec} multiply-add",
                "frac_of_sustained": ach / peak_sus, "sustained_peak": peak_sus,
                "algorithmic": f"2*n_nz*9n_pi*9m = {flops:.4g} flop per launch",
                "hardware_products": n_prod, "hardware_tflops": ach * n_prod,
                "tensor_pipe_peak": pk["bf16_tflops"] * ratio}
        if prec == "f64_emu":
            # operands' slices read once plus the FP64 nzdata written once
            roof["algorithmic_bytes"] = 7 * 2 * K * (tab.n_nz + 9 * n_tiles) + nz_bytes
    else:
        byts = scatter_bytes if dom == 2 else pull_bytes
        ach = byts / (stage_avg[dom] / 1e3) / 1e9
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_source": pk_kind}
    tr = NCU_TRAFFIC.get((roof["kernel"], workload, prec))
    if tr is not None and n_tiles != workload_config(workload)["tiles"]:
        tr = None          # captured on one launch over the whole workload, not this rank's slab and halo
    if tr is not None:
        if tr[2] == kernel_source_digest(roof["kernel"]):
            roof["traffic"] = tr[0]
            roof["traffic_source"] = tr[1]
        else:
            roof["traffic_stale"] = f"{tr[1]} was captured from an earlier version of the kernel"
    roof["stages_ms"] = dict(zip(names, [round(float(x), 4) for x in stage_avg]))
    # the paper times the generation of the nonzero values (steps 1 and 3) without the scatter
    nz_ms = float(stage_avg[0] + stage_avg[1])
    roof["nonzeros_only"] = {"ms": round(nz_ms, 4), "tiles_per_s": n_tiles / (nz_ms / 1e3) if nz_ms > 0 else None}
    roof["scatter_gbs"] = scatter_bytes / (stage_avg[2] / 1e3) / 1e9
    roof["scatter_frac_hbm"] = roof["scatter_gbs"] / pk["hbm_gbs"]
    roof["scatter_algorithmic_bytes"] = scatter_bytes
    roof["pullback_gbs"] = pull_bytes / (stage_avg[0] / 1e3) / 1e9
    return roof


def time_form(plan, ctrl, prec, flush, stream, reps=3):
    """Median ms of `reps` flushed assemblies in precision `prec` (CUDA events), the output and the
    per-stage times of the last one."""
    import torch
    o = plan.assemble(ctrl, 1.0, 0.3, prec)
    torch.cuda.synchronize()
    tms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.assemble(ctrl, 1.0, 0.3, prec, out=o, stage_times=True)
        b.record(stream)
        torch.cuda.synchronize()
        tms.append(a.elapsed_time(b))
    st, _ = plan.stage_times()
    return statistics.median(tms), o, st


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.report:
        return run_report(args)

    import torch
    import paper_2107_09568_gb300 as msasm
    import synth

    affinity = bind_to_gpu_local_cpus(local)      # before any pinned host buffer exists
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    msasm.load()

    w = synth.workload(args.workload)
    macro, n_elem, n_total, t0, t1, t_halo = slab_setup(args.workload, world, rank)
    micro = synth.micro_cross(w.n_e, w.width)
    tab = msasm.Tables(micro, w.q)
    plan = msasm.Plan(tab, macro, max_tiles_per_pass=(t_halo - t0) if world > 1 else 0)
    r0, r1, v0, v1, _ = plan.range(t0, t1)
    ctrl = torch.tensor(macro.ctrl, dtype=torch.float64, device="cuda")
    prec = args.precision
    out = torch.empty(v1 - v0, dtype=msasm.Plan.value_dtype(prec), device="cuda")     # this rank's rows
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()
    step = lambda **kw: plan.assemble_range(ctrl, t0, t1, 1.0, 0.3, prec, out=out, **kw)

    # correctness of the timed configuration: degenerate check (and the tensor-core pipeline flag)
    if world == 1:
        plan.assemble(ctrl, 1.0, 0.3, prec, out=out, check_degenerate=True)
    for _ in range(args.warmup):
        flush.zero_()
        step(stage_times=True)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    clocks.wait_first_sample()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_begin()
    stage_ms, launches = np.zeros(3), 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                                  # L2 flush between timed steps (not timed)
        ev[k][0].record(stream)
        step(stage_times=True)                         # the whole mesh at N = 1 (msasm_assemble's path)
        ev[k][1].record(stream)
        ms, ln = plan.stage_times()                    # events recorded inside the call, same stream
        stage_ms += np.array(ms)
        launches += sum(ln)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks.mark_end()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = whole_job_rate(t1 - t0, world, args.steps, total_ms)      # balanced ranges: equal tiles per rank
    vbytes = 8 if prec in ("f64", "f64_emu") else 4
    stiff_gbs = (v1 - v0) * vbytes * world * args.steps / (total_ms / 1e3) / 1e9

    # end to end through the public C ABI with host buffers (copies inside the timed region), on
    # every rank; the job's rate is set by the slowest rank
    e2e = None
    if not args.no_e2e:
        h_ctrl = torch.tensor(macro.ctrl, dtype=torch.float64).pin_memory()
        h_vals = torch.empty(v1 - v0, dtype=msasm.Plan.value_dtype(prec)).pin_memory()
        if world == 1:       # msasm_assemble_host: control net in, values out, copies overlapped with passes
            e_step = lambda: plan.assemble_host(h_ctrl, h_vals, 1.0, 0.3, prec)
            api = "msasm_assemble_host (pinned host buffers)"
        else:                # msasm_assemble_range on this rank's slab, with the copies around it
            def e_step():
                ctrl.copy_(h_ctrl, non_blocking=True)
                step()
                h_vals.copy_(out, non_blocking=True)
                torch.cuda.synchronize()
            api = "H2D control net, msasm_assemble_range, D2H of the rank's values (pinned host buffers)"
        e_step()
        e_steps = max(3, min(args.steps, 9))
        if dist is not None:
            dist.barrier()
        e_ms = []
        for _ in range(e_steps):
            flush.zero_(); torch.cuda.synchronize()
            ts = time.perf_counter()
            e_step()
            e_ms.append(1e3 * (time.perf_counter() - ts))
        # the median step: the host link shows occasional slow transfers (a step of 116-149 ms among
        # 70 ms ones on the 4000-tile beam), which the mean would fold into the rate
        em = max_over_ranks(statistics.median(e_ms), dist, "cuda")
        e2e = {"value": whole_job_rate(t1 - t0, world, 1, em), "unit": "tiles/s", "ms_per_step": em,
               "steps": e_steps, "statistic": "median of the steps", "ms_mean": sum(e_ms) / e_steps,
               "h2d_bytes_per_step": int(h_ctrl.numel() * 8) * world,
               "d2h_bytes_per_step": int((v1 - v0) * vbytes) * world, "api": api, "host_cpus": affinity}
        del h_vals, h_ctrl

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    pk, pk_kind = peaks()
    stage_avg = stage_ms / args.steps
    if world > 1:
        # rank 0's kernels: its slab plus the halo layer, writing its own rows
        roof = roofline_of(stage_avg, prec, tab, t_halo - t0, v1 - v0, pk, pk_kind, args.workload)
        line = {"metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": dict(workload_config(args.workload), mesh=list(n_elem), tiles=n_total,
                               tiles_per_gpu=t1 - t0),
                "execution": f"one mesh split into {world} contiguous tile slabs, one per GPU; each rank "
                             "recomputes the layer of tiles above its slab (halo) and writes only its own rows",
                "sizes": {"rank0_rows": r1 - r0, "rank0_values": v1 - v0, "rank0_tiles_with_halo": t_halo - t0},
                "stiffness_gbs": stiff_gbs, "roofline": roof, "cpu_baseline": None, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "forms": "reported at N = 1",
                "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return 0
    roof = roofline_of(stage_avg, prec, tab, plan.n_tiles, plan.nnz, pk, pk_kind, args.workload)

    # every precision form on the same workload: throughput and relative Frobenius error against the
    # plain FP64 GPU form (the CUDA-core DFMA contraction)
    forms = {}
    if prec == "f64":
        ref64 = out.clone()
    else:
        ms64, ref64, st64 = time_form(plan, ctrl, "f64", flush, stream, reps=2)
        forms["f64"] = {"tiles_per_s": plan.n_tiles / (ms64 / 1e3), "ms": ms64,
                        "stiffness_gbs": plan.nnz * 8 / (ms64 / 1e3) / 1e9, "rel_fro_vs_f64_gpu": 0.0,
                        "stages_ms": [round(x, 4) for x in st64], "note": "the plain FP64 GPU form"}
    main_err = None
    if prec != "f64":
        main_err = (torch.linalg.vector_norm(out.double() - ref64) / torch.linalg.vector_norm(ref64)).item()
    for f in [x for x in args.forms.split(",") if x and x not in forms]:
        if f == prec:
            forms[f] = {"tiles_per_s": value, "ms": total_ms / args.steps, "stiffness_gbs": stiff_gbs,
                        "rel_fro_vs_f64_gpu": main_err if main_err is not None else 0.0,
                        "stages_ms": [round(float(x), 4) for x in stage_avg], "note": "the headline (timed above)"}
            continue
        try:
            ms, o, st = time_form(plan, ctrl, f, flush, stream)
            err = (torch.linalg.vector_norm(o.double() - ref64) / torch.linalg.vector_norm(ref64)).item()
            forms[f] = {"tiles_per_s": plan.n_tiles / (ms / 1e3), "ms": ms,
                        "stiffness_gbs": plan.nnz * o.element_size() / (ms / 1e3) / 1e9, "rel_fro_vs_f64_gpu": err,
                        "stages_ms": [round(x, 4) for x in st]}
            del o
        except msasm.MsasmError as e:
            forms[f] = {"unavailable": str(e)}
    if "f64" in forms:
        for f, v in forms.items():
            if "ms" in v:
                v["speedup_vs_f64_gpu"] = forms["f64"]["ms"] / v["ms"]
    del ref64
    sizes = {"nnz": plan.nnz, "rows": plan.n_rows, "n_nz": tab.n_nz, "n_pi": tab.n_pi,
             "values_gb": plan.nnz * vbytes / 1e9}
    n_tiles = plan.n_tiles
    del out, plan, tab
    torch.cuda.empty_cache()

    # the other two lattice workloads, each against the plain FP64 GPU form: the learned surrogate of
    # the graded quarter arc (2000 tiles) and the adjoint gradient of the cantilever plate (2000 tiles)
    extra = {}
    if not args.no_extra:
        from paper_2107_09568_gb300 import workloads as wl
        t0 = time.perf_counter()
        extra["surrogate_arc2000"] = wl.surrogate(flush)
        extra["surrogate_arc2000"]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        a = wl.adjoint(flush, cg_tol=1e-6, fd_precision="f64")
        a["forms"] = {f: {"grad_ms": a[f"grad_ms_{f}"],
                          "rel_l2_vs_f64_gpu": 0.0 if f == "f64" else a[f"grad_rel_{f}_vs_f64"],
                          "speedup_vs_f64_gpu": a["grad_ms_f64"] / a[f"grad_ms_{f}"]}
                      for f in ("f64", "f64_emu", "f32")}
        a["wall_s"] = time.perf_counter() - t0
        extra["adjoint_cantilever2000"] = a
        torch.cuda.empty_cache()
        # the matrix-free product (Sec. 4.2) on the 1000-tile beam against the CSR product of the
        # assembled matrix: the split forms apply the tile blocks in the contraction's epilogue
        t0 = time.perf_counter()
        extra["linop_beam1000"] = wl.linop(flush)
        extra["linop_beam1000"]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu:
        prob = oracle_problem(args.workload)
        dt, n = cpu_reference_time(prob, 400 if n_tiles >= 1000 else n_tiles)
        cpu = {"value": n / dt, "unit": "tiles/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"{n} random tiles of the workload, FP64 lookup form (pullback, contraction, "
                         f"scatter ordering), {dt:.1f} s"}

    line = {"metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": workload_config(args.workload),
            "execution": "one GPU: the whole mesh (msasm_assemble_range over all tiles, the path of msasm_assemble)",
            "sizes": sizes, "stiffness_gbs": stiff_gbs, "rel_fro_vs_f64_gpu": main_err, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "forms": forms,
            "workloads": extra, "wall_s_timed_region": wall}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
