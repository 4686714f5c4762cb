"""Benchmark of the coupled platelet fluid-structure step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

One step = one pass of the whole hot path (membrane forces + wall term, bond
forces, spreading, lattice Boltzmann, interpolation + advection, adhesion
update) on the full-scale workload: a 512x256x256 D3Q19 Couette channel
(33.5 M cells) at wall shear 3000/s (tau = 0.8), 500 platelets of 2562
membrane nodes + 800 SCE elements with 5000 receptor sites each, ligands on
the whole bottom wall.  Inputs are synthetic and seeded.  The state (~7 GB)
is far larger than the 126 MB L2, so no flush is needed between steps; the
K timed steps run back to back through sim_step and are timed with CUDA
events on the launching stream.  `value` is the plain FP32 form; the
16-bit-storage and surrogate forms run beside it on the same workload.
The 128x64x64 channel (10 platelets; its state fits in L2, so L2 is flushed
before each of its steps) is reported as a secondary line.

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload on its own GPU (independent chambers: weak scaling,
no data-path collective); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS + membrane-node updates/s, % HBM roofline, vs plain FP32"
WORKLOAD = ("full scale 512x256x256 D3Q19 Couette channel (33.5 M cells), shear 3000/s, tau 0.8; 500 platelets x "
            "(2562 membrane nodes + 800 SCE), 5000 receptor sites each, ligands on the whole bottom wall; plain "
            "FP32 populations (FP64 positions)")
CHANNEL = ("channel 128x64x64 D3Q19 Couette, shear 1000/s, tau 0.8; 10 platelets x (2562 membrane nodes "
           "+ 800 SCE), 5000 receptor sites each, ligand patch 64x32; plain FP32 (FP64 positions)")
# accelerated adhesion kinetics (lattice units) of the full-scale comparison of
# the storage and membrane forms, so that bonds form within the timed window
FAST_KINETICS = dict(kon0_dt=0.05, koff0_dt=0.005, sigma=0.02, kT=0.05, gamma=0.05)
LB_BYTES_PER_CELL = 152          # 19 float loads + 19 float stores
LB_BYTES_PER_CELL_MIXED = 108    # 19 16-bit f^neq + one float4 (v, rho - 1), each read and written
# per step: membrane elements, coef, nodes, bond forces, spread, lb, interp,
# out-of-reach platelets, rupture, propose, resolve; plus the hi/lo split of X
# once per graph launch (the interpolation prepares it for the other steps)
KERNELS_PER_STEP = 11


def graph_launches(n):
    """Graph launches of sim_step(n): eight-step graphs while eight steps
    remain, then four-step ones, then single steps."""
    g = 0
    while n >= 4:
        n -= 8 if n >= 8 else 4
        g += 1
    return g + n


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def lb_kernel_sha():
    """Hash of the FP32 lattice kernel's source: the on-site wall helper it
    calls (csrc/pfsi_internal.cuh), its per-cell body fp32_cell and the
    kernel k_lb_step (csrc/lb.cu); the rest of those files does not change
    the kernel the traffic figure was measured on."""
    csrc = os.path.join(ROOT, "paper_1312_2234_b300", "csrc")
    hdr = open(os.path.join(csrc, "pfsi_internal.cuh")).read()
    a = hdr.index("template <int s>\n__device__ __forceinline__ void onsite_wall")
    b = hdr.index("\n}\n", a) + 3
    src = open(os.path.join(csrc, "lb.cu")).read()
    c = src.index("__device__ __forceinline__ void fp32_cell(")
    c2 = src.index("__global__ void __launch_bounds__(kMaxRowBlock) k_lb_step(")
    d = src.index("\n}\n", c2) + 3
    return hashlib.sha256((hdr[a:b] + src[c:d]).encode()).hexdigest()[:16]


def ncu_traffic(name="lb_step_full_512x256x256.md"):
    """DRAM bytes per launch of the lattice kernel from a committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    sh = re.search(r"lb_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not sh or sh.group(1) != lb_kernel_sha():
        return None
    return float(m.group(1))


class L2Flush:
    """Evicts the 126 MB L2 between timed steps: writes a 512 MB buffer, then
    (unless write_only) reads a 256 MB one, so that the L2 ends up holding
    clean lines of an unrelated buffer.  A write alone leaves ~126 MB of
    dirty lines whose write-backs the next step's first heavy kernel pays
    (the channel step reads ~4 us slower that way)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.sink = torch.empty(1, dtype=torch.float32, device=dev)

    def __call__(self, k=0, write_only=False):
        import torch
        self.w.fill_(float(k))
        if not write_only:
            torch.sum(self.r, dim=0, keepdim=True, out=self.sink)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)
        return False

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, ws


def reduce_max(x: float, ws: int) -> float:
    """Maximum of a per-rank scalar over all ranks (identity for one rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


SAMPLE = ("1/16 of the full-scale channel along x: 32x256x256 cells (2.1 M), 31 platelets of the same kind "
          "(2562 + 800 SCE, 5000 receptor sites each) at the same density, shear 3000/s, ligands on the whole "
          "bottom wall (workload.config_full_sample)")


def cpu_baseline(threads):
    """The oracle as it stands on a bounded sample of the workload (SAMPLE):
    one coupled step after one untimed step, once on all host cores (its
    loops over independent cells and nodes run on OpenMP threads; the rest
    is serial) and once on one core."""
    import oracle
    from paper_1312_2234_b300 import workload
    w = workload.config_full_sample(seed=0)
    sim = oracle.Sim(w)
    oracle.set_threads(threads)
    sim.step()                      # untimed first step
    N = w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"]
    legs = {}
    for n in (threads, 1):
        oracle.set_threads(n)
        t0 = time.perf_counter()
        sim.step()
        legs[n] = time.perf_counter() - t0
    oracle.set_threads(threads)
    dt = legs[threads]
    return {"value": N / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": "%s: one coupled step after one untimed step, %.2f s on %d threads (OpenMP over the "
                      "lattice cells and the interpolated nodes; membrane, spreading and bonds serial)"
                      % (SAMPLE, dt, threads),
            "node_updates_per_s": w["M"] / dt,
            "single_thread": {"value": N / legs[1] / 1e6, "unit": "MLUPS", "cores": 1,
                              "seconds_per_step": legs[1], "node_updates_per_s": w["M"] / legs[1]},
            "nproc": os.cpu_count()}


def run_reference(args, rank, ws):
    """The oracle on the host cores (OpenMP over all of them) on the native
    arm's workload, metric and unit: each step one coupled oracle step of a
    bounded sample of the workload (SAMPLE)."""
    from paper_1312_2234_b300 import workload
    import oracle
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    w = workload.config_full_sample(seed=0)
    N = w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"]
    sim = oracle.Sim(w)
    for _ in range(args.warmup):
        sim.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step()
    dt = time.perf_counter() - t0
    val = N * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": SAMPLE, "cells": N, "nodes": w["M"],
                                            "parallelism": "%d host threads (OpenMP)" % threads},
            "node_updates_per_s": w["M"] * args.steps / dt,
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": "%s; %d coupled steps after %d untimed" % (SAMPLE, args.steps, args.warmup)},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args, rank, ws):
    import torch
    from paper_1312_2234_b300 import fsi, workload

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t_build = time.perf_counter()
    w = workload.config_full(seed=0)
    log("full-scale workload built in %.1f s" % (time.perf_counter() - t_build))
    g = w["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    M = w["M"]
    sim = fsi.Simulation(w, device=dev)
    sim.step(args.warmup)
    torch.cuda.synchronize()

    # the timed region: K steps back to back (sim_step replays eight-step
    # graphs, then four-step and single-step ones); the ~7 GB state does not
    # fit in L2, so consecutive steps re-read it from HBM
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        sim.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    total_s = reduce_max(start.elapsed_time(end) / 1e3, ws)
    ms_per_step = 1e3 * total_s / args.steps

    # the same steps one graph launch each, timed one by one (no overlap of
    # one step's adhesion update with the next step's membrane pass)
    single_ms = []
    for _ in range(args.steps):
        a_ev = torch.cuda.Event(enable_timing=True)
        b_ev = torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        fsi.sim_step(sim.h, 1)
        b_ev.record(stream)
        b_ev.synchronize()
        single_ms.append(a_ev.elapsed_time(b_ev))

    # the dominant kernel where it runs: the same single steps with two CUDA
    # events recorded around the lattice kernel inside the step graph
    fsi.sim_time_lb(sim.h, True)
    lb_ms = []
    for _ in range(max(args.steps, 10)):
        sim.step(1)
        lb_ms.append(fsi.sim_lb_ms(sim.h))
    fsi.sim_time_lb(sim.h, False)
    # the average launch duration (the event timer ticks in ~1 us steps)
    lb_s = statistics.fmean(lb_ms) / 1e3
    lb_bytes = LB_BYTES_PER_CELL * N
    peaks = measured_peaks()
    if peaks:
        peak, peak_note = peaks["hbm_gbs"], "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    else:
        peak, peak_note = 6400.0, "fallback 6.4 TB/s"
    achieved = lb_bytes / lb_s / 1e9
    traffic = ncu_traffic()
    e2e = run_e2e(args, w, sim, dev, stream, ws)
    del sim
    torch.cuda.empty_cache()

    channel, sim_c, w_c = run_channel(args, dev, stream, ws)
    extras = {"channel": channel}
    forms = {}
    if not args.no_extras:
        flush = L2Flush(dev)
        extras["fem_bending"] = run_fem(args, w_c, channel["ms_per_step"], dev, flush, stream, w)
        extras["platelet_pair"] = run_pair(args, dev, flush, stream)
        del flush
        torch.cuda.empty_cache()
        extras["batched"] = run_batched(args, dev, stream)
        extras["surrogate"], sg_params = run_surrogate(args, w_c, sim_c, dev, stream)
        del sim_c
        torch.cuda.empty_cache()
        if not args.no_mixed:
            forms = run_forms(args, w, dev, stream, sg_params, ws)

    if rank != 0:
        return
    base = cpu_baseline(os.cpu_count() or 1) if args.cpu_steps > 0 else None
    value = ws * N * args.steps / total_s / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": N, "nodes": M, "sites": int(len(w["sites"]["tri"])),
                   "ligands": int(w["bonds"]["lig_ni"] * w["bonds"]["lig_nj"]),
                   "l2": "no flush: the state (~7 GB of populations, fields and platelets) is far larger than "
                         "the 126 MB L2",
                   "parallelism": "replicas",
                   "graph": "sim_step(K): eight-step CUDA graphs (each step's adhesion update beside the next "
                            "step's membrane pass), then four-step and single-step graphs",
                   "single_step_graph_ms": statistics.fmean(single_ms)},
        "node_updates_per_s": ws * M * args.steps / total_s,
        "roofline": {"bound": "hbm", "kernel": "k_lb_step", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note,
                     "algorithmic_bytes_per_launch": lb_bytes, "launch_ms": 1e3 * lb_s,
                     "launch_ms_median": statistics.median(lb_ms),
                     "timing": "mean over %d single steps of CUDA events recorded around the kernel inside "
                               "the step graph (includes the graph's event-node latency)" % len(lb_ms)},
        "lb_share_of_step": (1e3 * lb_s) / statistics.fmean(single_ms),
        "mixed_precision": forms,
        "configurations": extras,
        "cpu_baseline": base,
        "e2e": e2e,
        "gpu_launches": KERNELS_PER_STEP * args.steps + graph_launches(args.steps),
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def run_e2e(args, w, sim, dev, stream, ws):
    """End to end through the public API with host buffers: the node
    positions come from pinned host memory and the developed flow is set up
    on the device inside the timed region, then sim_step_track steps the
    simulation and copies every step's platelet centroids to pinned host
    memory; and the same steps with all node positions of every step copied
    to the host (sim_step_record)."""
    import torch
    g = w["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    M = w["M"]
    lat = sim.lattice
    hostX = torch.from_numpy(np.ascontiguousarray(w["X"])).pin_memory()
    nplt = int(w["mesh"]["n_plt"])
    cbuf = torch.empty(72 * nplt, dtype=torch.float64, device=dev)
    # instantiate the tracked graphs (both eight-step slot groups and the single steps)
    sim.step_track(18, cbuf, torch.empty(18, 3 * nplt, dtype=torch.float64).pin_memory())
    out = torch.empty(args.steps, 3 * nplt, dtype=torch.float64).pin_memory()
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.X.copy_(hostX, non_blocking=True)   # the platelets' state comes from the host
        lat.init_shear()                         # the flow is set up on the device
        sim.step_track(args.steps, cbuf, out)
        t1.record(stream)
        t1.synchronize()
        runs.append(t0.elapsed_time(t1) / 1e3)
    e2e_s = reduce_max(statistics.median(runs), ws)
    h2d = hostX.numel() * 8 / args.steps
    ring = 4
    dev_ring = torch.empty(ring, 3 * M, dtype=torch.float64, device=dev)
    outX = torch.empty(ring, 3 * M, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t2 = torch.cuda.Event(enable_timing=True)
    t3 = torch.cuda.Event(enable_timing=True)
    t2.record(stream)
    sim.step_record(args.steps, dev_ring, outX)
    t3.record(stream)
    t3.synchronize()
    pos_s = reduce_max(t2.elapsed_time(t3) / 1e3, ws)
    return {"value": ws * N * args.steps / e2e_s / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(3 * nplt * 8),
            "note": "node positions uploaded from pinned memory and the developed flow initialised on the "
                    "device inside the timed region (upload bytes amortised per step); every step's "
                    "platelet centroids read back to pinned host memory; one continuous run of the timed "
                    "steps; median of three such runs",
            "with_positions_every_step": {
                "value": ws * N * args.steps / pos_s / 1e6, "unit": "MLUPS",
                "d2h_bytes_per_step": int(3 * M * 8),
                "d2h_gbs": 3 * M * 8 * args.steps / pos_s / 1e9,
                "note": "all node positions of every step copied to pinned host memory on a second "
                        "stream (sim_step_record); the device-to-host link bounds it"}}


def run_channel(args, dev, stream, ws):
    """The 128x64x64 channel with 10 platelets: L2 flushed before every
    step (its state fits in L2), single steps timed with CUDA events; its
    lattice kernel's roofline (L2-resident writes), and the same workload
    on 16-bit population storage with its deviation from this FP32 run."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    w = workload.config_channel(seed=0)
    g = w["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    sim = fsi.Simulation(w, device=dev)
    flush = L2Flush(dev)
    for _ in range(args.warmup):
        flush(1)
        sim.step(1)
    torch.cuda.synchronize()
    ms = []
    for k in range(args.steps):
        flush(k)
        a_ev = torch.cuda.Event(enable_timing=True)
        b_ev = torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        sim.step(1)
        b_ev.record(stream)
        b_ev.synchronize()
        ms.append(a_ev.elapsed_time(b_ev))
    step_ms = statistics.fmean(ms)
    snap = {"X": sim.X.cpu().numpy(), "U": sim.U.cpu().numpy(),
            "bound": sim.bonds.bound.cpu().numpy() if sim.bonds else None}
    fsi.sim_time_lb(sim.h, True)
    lb_ms = []
    for k in range(max(args.steps, 10)):
        flush(k)
        sim.step(1)
        lb_ms.append(fsi.sim_lb_ms(sim.h))
    fsi.sim_time_lb(sim.h, False)
    lb_s = statistics.fmean(lb_ms) / 1e3
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = LB_BYTES_PER_CELL * N / lb_s / 1e9
    mixed = {} if args.no_mixed else {s: run_mixed(args, w, s, dev, flush, stream, snap, ws)
                                      for s in ("bf16", "fp16")}
    out = {"workload": CHANNEL, "cells": N, "nodes": w["M"], "sites": int(len(w["sites"]["tri"])),
           "value": N * len(ms) / (sum(ms) / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": step_ms,
           "l2": "L2-resident state: flushed before every step (512 MB written, then 256 MB read)",
           "lb_kernel": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "launch_ms": 1e3 * lb_s, "traffic": ncu_traffic("lb_step_channel_128x64x64.md"),
                         "note": "L2-resident: the kernel's writes stay in the 126 MB L2"},
           "mixed_precision": {k: dict(v, vs_fp32=v["value"] / (N * len(ms) / (sum(ms) / 1e3) / 1e6))
                               for k, v in mixed.items()}}
    del flush
    torch.cuda.empty_cache()
    return out, sim, w


def run_mixed(args, w, storage, dev, flush, stream, snap, ws):
    """The coupled step with 16-bit f^neq lattice storage: value, step time,
    the lattice kernel's roofline, and the deviation from the FP32 run."""
    import torch
    from paper_1312_2234_b300 import fsi
    g = w["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    # launch shape of the 16-bit lattice kernel picked by the autotuner (as at full scale)
    sim = fsi.Simulation(w, device=dev, storage=storage, tune=True)
    for _ in range(args.warmup):
        flush(1)
        sim.step(1)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    for k in range(args.steps):
        flush(k)
        starts[k].record(stream)
        sim.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    total_s = reduce_max(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, ws)
    X0 = np.ascontiguousarray(w["X"])
    dX32 = snap["X"] - X0
    err = {"displacement_rel": float(np.abs(sim.X.cpu().numpy() - snap["X"]).max() / np.abs(dX32).max()),
           "node_velocity_rel": float(np.abs(sim.U.cpu().numpy() - snap["U"]).max() / np.abs(snap["U"]).max())}
    if snap["bound"] is not None:
        b = sim.bonds.bound.cpu().numpy()
        err["bonds_fp32"] = int((snap["bound"] >= 0).sum())
        err["bonds"] = int((b >= 0).sum())
        err["sites_differing"] = int((b != snap["bound"]).sum())
    fsi.sim_time_lb(sim.h, True)
    lb_ms = []
    for k in range(max(args.steps, 10)):
        flush(k)
        sim.step(1)
        lb_ms.append(fsi.sim_lb_ms(sim.h))
    fsi.sim_time_lb(sim.h, False)
    # the average launch duration (the event timer ticks in ~1 us steps, so
    # the mean of many intervals also resolves below one tick)
    lb_s = statistics.fmean(lb_ms) / 1e3
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = LB_BYTES_PER_CELL_MIXED * N / lb_s / 1e9
    return {"value": ws * N * args.steps / total_s / 1e6, "unit": "MLUPS",
            "ms_per_step": 1e3 * total_s / args.steps, "fp16_exponent": int(sim.lattice.p.fp16_exponent),
            "lb_kernel": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                          "algorithmic_bytes_per_launch": LB_BYTES_PER_CELL_MIXED * N, "launch_ms": 1e3 * lb_s},
            "error_vs_fp32_after_%d_steps" % (args.warmup + args.steps): err}


def timed_steps(step, steps, stream):
    """Device time of `steps` calls of step() (CUDA events, after a sync)."""
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def run_batched(args, dev, stream):
    """64 independent chambers of uneven sizes (48..128 per side), one
    platelet each: stepped one chamber at a time (one graph launch per
    chamber), then as one batch (one graph launch for all chambers per step,
    every kernel of the step one launch for all 64 chambers; the lattice
    update one persistent launch per storage mode, its column shapes and
    grid tuned), with FP32 populations and with 16-bit f^neq storage.  The
    lattice-only batched step (lb_batch_step on the 64 lattices) is timed
    too, against the HBM roofline."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    ws_ = workload.config_batched(seed=0)
    cells = sum(w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"] for w in ws_)
    nodes = sum(w["M"] for w in ws_)
    steps, warm = max(3, args.steps // 5), 3
    out = {"workload": "64 chambers, sides 48..128, shear 500..3000/s, 2000..25000 receptors, stiffness x0.5..2, "
                       "one platelet (2562 + 800 SCE) each", "cells": cells, "nodes": nodes, "steps": steps,
           "l2": "working set far above L2 (no flush)"}
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    for storage in ("fp32", "bf16", "fp16"):
        sims = [fsi.Simulation(w, device=dev, storage=storage) for w in ws_]
        if storage == "fp32":
            for _ in range(warm):
                for sm in sims:
                    sm.step(1)
            t = timed_steps(lambda: [sm.step(1) for sm in sims], steps, stream)
            out["fp32_one_launch_per_chamber"] = {"value": cells * steps / t / 1e6, "unit": "MLUPS",
                                                  "ms_per_step": 1e3 * t / steps}
        batch = fsi.Batch(sims, steps_per_graph=1, tune=True)
        batch.step(warm)
        t = timed_steps(lambda: batch.step(1), steps, stream)
        out[storage + "_batched"] = {"value": cells * steps / t / 1e6, "unit": "MLUPS", "ms_per_step": 1e3 * t / steps,
                                     "node_updates_per_s": nodes * steps / t}
        del batch, sims
        torch.cuda.empty_cache()
        # the lattice update alone: the same 64 lattices in one LatticeBatch
        lats = [fsi.Lattice(w["grid"]["nx"], w["grid"]["ny"], w["grid"]["nz"], w["grid"]["tau"], w["grid"]["u_top"],
                            device=dev, storage=storage) for w in ws_]
        for lat in lats:
            lat.init_shear()
        lb = fsi.LatticeBatch(lats)
        lb.autotune(reps=3)
        lb.step(warm)
        t = timed_steps(lambda: lb.step(1), steps, stream)
        per_cell = LB_BYTES_PER_CELL if storage == "fp32" else LB_BYTES_PER_CELL_MIXED
        gbs = per_cell * cells / (t / steps) / 1e9
        out[storage + "_lattice_batch"] = {"value": cells * steps / t / 1e6, "unit": "MLUPS",
                                           "ms_per_step": 1e3 * t / steps, "bytes_per_cell": per_cell,
                                           "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak}
        if storage != "fp32":
            shp = lb.shapes()
            out[storage + "_lattice_batch"]["shapes"] = {n: shp.count(i) for i, n in
                                                         enumerate(("pair 64x4", "32x4", "16x8"))}
        del lb, lats
        torch.cuda.empty_cache()
    return out


def run_batched_only(args):
    import torch
    torch.cuda.init()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    print(json.dumps(run_batched(args, dev, stream)))


def run_surrogate(args, w_channel, sim_channel, dev, stream):
    """The learned membrane surrogate: trained on the channel's own trajectory
    (its current state plus perturbed copies), then the 256x128x128 channel
    with 100 platelets stepped with the plain membrane solver and with the
    surrogate (plain solver kept as the judge of its force error)."""
    import time as _t
    import torch
    from paper_1312_2234_b300 import fsi, surrogate, workload
    rng = np.random.default_rng(0)
    m = w_channel["mesh"]
    t0 = _t.perf_counter()
    params = fsi.SurrogateParams(device=dev)
    params.set(surrogate.init_params(rng))
    sg_c = fsi.Surrogate(m, "bf16", device=dev)
    # trajectory snapshots of the channel (every 200 steps over 2000 more
    # steps of the plain method), each with a few perturbed copies
    snaps = [w_channel["X"]]
    for _ in range(10):
        sim_channel.step(200)
        snaps.append(sim_channel.X.cpu().numpy())
    states = surrogate.perturbed_states(snaps, m, amplitudes=(0.0003, 0.003), copies=2, rng=rng)
    data = surrogate.prepare(sg_c, params, w_channel["membrane"], states)
    train_steps = 4000
    hist = surrogate.train(params, data, train_steps, batch=4096, lr=2e-3, log_every=500)
    torch.cuda.synchronize()
    t_train = _t.perf_counter() - t0
    w4 = workload.config_surrogate(seed=0)
    N = w4["grid"]["nx"] * w4["grid"]["ny"] * w4["grid"]["nz"]
    steps, warm = max(3, args.steps // 5), 3
    out = {"workload": "256x128x128 channel, shear 1500/s, 100 platelets x 2562 nodes", "cells": N,
           "nodes": w4["M"], "steps": steps,
           "training": {"samples": len(data), "steps": train_steps, "batch": 4096, "seconds": t_train,
                        "loss_first": hist[0][1], "loss_last": hist[-1][1],
                        "data": "channel trajectory (11 snapshots over 2000 steps of the plain method) + 2 "
                                "Gaussian perturbations of 0.03 % and of 0.3 % of the mean edge per snapshot; "
                                "targets: the plain local terms' element stresses at those states"}}
    sg4 = fsi.Surrogate(w4["mesh"], "bf16", device=dev)
    plain = fsi.Membrane(w4["membrane"], w4["mesh"], device=dev)
    after = 500      # steps after the timed ones: the flow deforms the platelets
    final = {}
    for mode in ("plain", "surrogate"):
        sim = fsi.Simulation(w4, device=dev)
        if mode == "surrogate":
            fsi.sim_set_surrogate(sim, sg4, params)
        sim.step(warm)
        t = timed_steps(lambda: sim.step(1), steps, stream)
        out[mode] = {"value": N * steps / t / 1e6, "unit": "MLUPS", "ms_per_step": 1e3 * t / steps,
                     "node_updates_per_s": w4["M"] * steps / t}
        sim.step(after)
        final[mode] = (sim.X.clone(), sim.U.clone())
        if mode == "surrogate":
            Fp = torch.zeros(3 * w4["M"], device=dev)
            Fs = torch.zeros_like(Fp)
            Fl = torch.zeros_like(Fp)
            plain.forces(sim.X, Fp)
            sg4.forces(params, plain, sim.X, Fs)
            fsi.Membrane(surrogate.local_params(w4["membrane"]), w4["mesh"], device=dev).forces(sim.X, Fl)
            mask = torch.as_tensor(np.asarray(w4["mesh"]["is_membrane"]).astype(bool), device=dev)
            X0 = torch.as_tensor(w4["X"], device=dev)
            (Xp, Up), (Xs, Us) = final["plain"], final["surrogate"]
            out["force_error"] = {
                "local_max_rel": surrogate.rel_force_error(Fs - Fp + Fl, Fl, mask),
                "total_max_rel": surrogate.rel_force_error(Fs, Fp, mask),
                "note": "surrogate vs plain membrane force on the surrogate run's state after %d steps; local = "
                        "springs + local area + bending, total adds the exact global terms" % (warm + steps + after)}
            out["run_error"] = {
                "velocity_max_rel": float((Us - Up).abs().max() / Up.abs().max()),
                "displacement_max_rel": float(((Xs - X0) - (Xp - X0)).abs().max() / (Xp - X0).abs().max()),
                "note": "node velocities and displacements of the surrogate run against the plain run after %d "
                        "steps from the same state" % (warm + steps + after)}
            out["membrane_us"] = {
                "plain": 1e6 * timed_steps(lambda: plain.forces(sim.X, Fp), 20, stream) / 20,
                "surrogate": 1e6 * timed_steps(lambda: sg4.forces(params, plain, sim.X, Fs), 20, stream) / 20}
        del sim
    out["vs_plain"] = out["surrogate"]["value"] / out["plain"]["value"]
    return out, params


def run_fem(args, w, ms_dihedral, dev, flush, stream, w_full=None):
    """The channel's coupled step with the finite-element bending of Eq. 6-10
    in place of the dihedral term (timed like the headline: L2 flushed before
    every step), and the bending term alone on the channel's and on the full
    scale's meshes (10 and 500 platelets of 1280 six-node elements)."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    wf = dict(w, membrane=dict(w["membrane"], bending="fem"))
    sim = fsi.Simulation(wf, device=dev)
    N = w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"]
    steps = max(3, args.steps)
    sim.step(3)
    ms = []
    for k in range(steps):
        flush(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(1)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    step_ms = float(np.mean(ms))
    out = {"workload": "channel 128x64x64, 10 platelets: coupled step with finite-element bending",
           "coupled": {"value": N / step_ms / 1e3, "unit": "MLUPS", "ms_per_step": step_ms,
                       "vs_dihedral": ms_dihedral / step_ms}}
    del sim
    if w_full is None:
        w_full = workload.config_full(seed=0)
    for name, wk in (("channel_mesh", w), ("full_scale_mesh", w_full)):
        fb = fsi.FemBending(wk["mesh"], device=dev)
        X = torch.as_tensor(np.ascontiguousarray(wk["X"], dtype=np.float64), device=dev)
        F = torch.zeros(3 * wk["M"], dtype=torch.float32, device=dev)
        for _ in range(3):
            fb.forces(1e-3, X, F)
        reps = 20
        t = timed_steps(lambda: fb.forces(1e-3, X, F), reps, stream)
        ne = int(np.asarray(wk["mesh"]["elem6"]).size // 6)
        out[name] = {"elements": ne, "us_per_evaluation": 1e6 * t / reps, "launches": 8,
                     "elements_per_s": ne * reps / t}
        del fb, X, F
        torch.cuda.empty_cache()
    return out


def run_pair(args, dev, flush, stream):
    """Two stacked platelets over the ligand patch (the platelet-platelet
    study): the coupled step with wall bonds and platelet-platelet bridges,
    and without the bridges, timed like the headline (L2 flushed before every
    step)."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    w = workload.config_pair(seed=0)
    N = w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"]
    out = {"workload": "64x48x40 channel, shear 1000/s, two stacked platelets (2562 + 800 SCE, 5000 receptors "
                       "each), wall bonds + platelet-platelet bridges", "cells": N, "nodes": w["M"],
           "sites": int(len(w["sites"]["tri"]))}
    steps = max(3, args.steps)
    for name, wk in (("with_bridges", w), ("without_bridges", {k: v for k, v in w.items() if k != "bridges"})):
        sim = fsi.Simulation(wk, device=dev)
        sim.step(3)
        ms = []
        for k in range(steps):
            flush(k)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        step_ms = float(np.mean(ms))
        out[name] = {"value": N / step_ms / 1e3, "unit": "MLUPS", "ms_per_step": step_ms}
        del sim
    out["bridge_us_per_step"] = 1e3 * (out["with_bridges"]["ms_per_step"] - out["without_bridges"]["ms_per_step"])
    return out


def run_forms(args, w, dev, stream, sg_params, ws):
    """The full-scale workload in its storage and membrane forms, all at the
    accelerated adhesion kinetics FAST_KINETICS (so that bonds form within
    the window): plain FP32, BF16 and FP16 f^neq storage with the plain
    membrane, and BF16 storage with the learned surrogate (plain solver for
    the global terms).  Each form runs W + K steps from the same state, the
    last K timed back to back; the 16-bit and surrogate forms are compared
    with the FP32 form after the same steps: node velocity and displacement,
    and the bond state (bond counts and sites whose state differs)."""
    import torch
    from paper_1312_2234_b300 import fsi
    g = w["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    wk = dict(w, bonds=dict(w["bonds"], **FAST_KINETICS))
    out = {"workload": WORKLOAD, "kinetics": dict(FAST_KINETICS, note="accelerated, lattice units"),
           "steps": args.steps, "warmup": args.warmup}
    ref = None
    X0 = np.ascontiguousarray(w["X"])
    for form in ("fp32", "bf16", "fp16", "bf16_surrogate"):
        storage = "fp32" if form == "fp32" else form.split("_")[0]
        sim = fsi.Simulation(wk, device=dev, storage=storage, tune=storage != "fp32")
        if form.endswith("surrogate"):
            sg = fsi.Surrogate(wk["mesh"], "bf16", device=dev)
            fsi.sim_set_surrogate(sim, sg, sg_params)
        sim.step(args.warmup)
        t = timed_steps(lambda: sim.step(args.steps), 1, stream)
        t = reduce_max(t, ws)
        X = sim.X.cpu().numpy()
        U = sim.U.cpu().numpy()
        bound = sim.bonds.bound.cpu().numpy()
        r = {"value": ws * N * args.steps / t / 1e6, "unit": "MLUPS", "ms_per_step": 1e3 * t / args.steps,
             "bonds": int((bound >= 0).sum())}
        if storage != "fp32":
            r["fp16_exponent" if storage == "fp16" else "shape"] = (
                int(sim.lattice.p.fp16_exponent) if storage == "fp16" else int(sim.shape))
        if ref is None:
            ref = (X, U, bound)
        else:
            dX = ref[0] - X0
            r["error_vs_fp32"] = {
                "node_velocity_rel": float(np.abs(U - ref[1]).max() / max(np.abs(ref[1]).max(), 1e-30)),
                "displacement_rel": float(np.abs(X - ref[0]).max() / max(np.abs(dX).max(), 1e-30)),
                "bonds_fp32": int((ref[2] >= 0).sum()), "bonds": r["bonds"],
                "bond_count_rel": abs(r["bonds"] - int((ref[2] >= 0).sum())) / max(int((ref[2] >= 0).sum()), 1),
                "sites_differing": int((bound != ref[2]).sum())}
        if form.endswith("surrogate"):
            r["surrogate_status"] = sg.status()
            del sg
        out[form] = r
        del sim
        torch.cuda.empty_cache()
    for form in ("bf16", "fp16", "bf16_surrogate"):
        out[form]["vs_fp32"] = out[form]["value"] / out["fp32"]["value"]
    return out


def run_full_only(args):
    """The full-scale step alone in its forms (profiling aid): plain FP32,
    16-bit storage and BF16 + surrogate with untrained surrogate weights
    (the same kernels and launch shapes as trained ones).  Prints one JSON
    line."""
    import torch
    from paper_1312_2234_b300 import fsi, surrogate, workload
    dev = torch.device("cuda", 0)
    params = fsi.SurrogateParams(device=dev)
    p = surrogate.init_params(np.random.default_rng(0))
    p["W3"] *= 1e-3     # a small untrained network keeps the run physical
    params.set(p)
    w = workload.config_full(seed=0)
    print(json.dumps({"kernel": "full-scale coupled step",
                      **run_forms(args, w, dev, torch.cuda.current_stream(), params, 1)}), flush=True)


def run_lb_only(args):
    """The lattice kernel alone on a grid of the caller's size (profiling aid:
    a grid larger than L2 makes its DRAM figures meaningful).  Prints one
    JSON line with its event-timed duration and algorithmic bandwidth."""
    import torch
    from paper_1312_2234_b300 import fsi

    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    lat = fsi.Lattice(nx, ny, nz, 0.8, (1e-3, 0.0, 0.0), storage=args.storage)
    if args.shape is not None:
        fsi.lb_set_shape(lat, args.shape)
    lat.init_shear()
    N = nx * ny * nz
    per_cell = LB_BYTES_PER_CELL if args.storage == "fp32" else LB_BYTES_PER_CELL_MIXED
    flush = L2Flush("cuda")
    small = per_cell * N < 2 * 126e6
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fsi.lb_step(lat.h, 1)
    ms = []
    for k in range(args.steps):
        if small:
            flush(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fsi.lb_step(lat.h, 1)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms) / 1e3
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    gbs = per_cell * N / t / 1e9
    print(json.dumps({"kernel": "k_lb_step", "storage": args.storage, "shape": fsi.lb_get_shape(lat), "grid": [nx, ny, nz],
                      "cells": N, "median_ms": 1e3 * t,
                      "min_ms": min(ms), "GLUPS": N / t / 1e9, "GBps": gbs, "peak_GBps": peak,
                      "frac": gbs / peak, "l2_flushed": small}), flush=True)


def run_surrogate_only(args):
    """The surrogate membrane force alone on the 256x128x128 channel's
    256,200 membrane nodes (profiling aid; untrained weights, which do not
    change the work): event-timed per call (the exact remainder of the plain
    passes and the fused tensor-core inference) against the plain membrane
    call."""
    import torch
    from paper_1312_2234_b300 import fsi, surrogate, workload
    w = workload.config_surrogate(seed=0)
    m = w["mesh"]
    n = w["M"]
    mem = fsi.Membrane(w["membrane"], m)
    sg = fsi.Surrogate(m, "bf16")
    params = fsi.SurrogateParams()
    params.set(surrogate.init_params(np.random.default_rng(0)))
    X = torch.as_tensor(w["X"] + 1e-3 * np.random.default_rng(1).standard_normal(w["X"].shape)).cuda()
    F = torch.zeros(3 * n, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sg.forces(params, mem, X, F)
        mem.forces(X, F)
    t_sg = timed_steps(lambda: sg.forces(params, mem, X, F), args.steps, stream) / args.steps
    t_plain = timed_steps(lambda: mem.forces(X, F), args.steps, stream) / args.steps
    flop = 2 * (64 * 128 + 144 * 128 + 144 * 32) * sg.rows
    print(json.dumps({"kernel": "k_sg_infer + exact global membrane terms", "nodes": n, "rows": sg.rows,
                      "surrogate_us": 1e6 * t_sg, "plain_us": 1e6 * t_plain,
                      "tensor_flop_per_call": flop, "status": sg.status()}), flush=True)


def run_fem_only(args):
    """The finite-element bending force alone (profiling aid): the 10-platelet
    channel mesh (12,800 six-node elements) or, with --grid 512x256x256, the
    full-scale mesh (640,000), event-timed per evaluation."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    w = workload.config_full(seed=0) if args.grid == "512x256x256" else workload.config_channel(seed=0)
    fb = fsi.FemBending(w["mesh"])
    X = torch.as_tensor(np.ascontiguousarray(w["X"], dtype=np.float64)).cuda()
    F = torch.zeros(3 * w["M"], device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fb.forces(1e-3, X, F)
    t = timed_steps(lambda: fb.forces(1e-3, X, F), args.steps, stream) / args.steps
    ne = int(np.asarray(w["mesh"]["elem6"]).size // 6)
    print(json.dumps({"kernel": "k_fem_elem + k_fem_node (8 launches) + k_fem_split", "elements": ne,
                      "nodes": w["M"], "us_per_evaluation": 1e6 * t, "elements_per_s": ne / t}), flush=True)


def run_bridges_only(args):
    """The platelet-platelet bridge update alone (profiling aid) on the
    two-stacked-platelet workload with raised kinetics (so that bridges form
    and break every step), the nodes held fixed; event-timed per update."""
    import torch
    from paper_1312_2234_b300 import fsi, workload
    w = workload.config_pair(seed=0)
    bp = dict(w["bridges"], sigma=0.02, kT=0.05, gamma=0.05, kon0_dt=0.3, koff0_dt=0.05)
    st = np.ascontiguousarray(w["sites"]["tri"], dtype=np.int32)
    sw = np.ascontiguousarray(w["sites"]["w"], dtype=np.float64).reshape(-1, 2)
    tri = torch.as_tensor(np.ascontiguousarray(w["mesh"]["tri"], dtype=np.int32).ravel()).cuda()
    bonds = fsi.Bonds(w["bonds"], st, sw, tri, w["bound"], w["lig_count"])
    br = fsi.Bridges(bp, bonds, w["mesh"]["node_plt"], w["mesh"]["n_plt"])
    X = torch.as_tensor(np.ascontiguousarray(w["X"], dtype=np.float64)).cuda()
    stream = torch.cuda.current_stream()
    state = {"k": 0}

    def one():
        br.step(X, state["k"])
        state["k"] += 1

    for _ in range(args.warmup):
        one()
    t = timed_steps(one, args.steps, stream) / args.steps
    ev = br.status()
    print(json.dumps({"kernel": "bridges_step (rupture, boxes, neighbours, candidate hash, choice, matching)",
                      "sites": int(len(st)), "us_per_update": 1e6 * t, "ruptures": ev[0], "formations": ev[1],
                      "standing": int((br.partner >= 0).sum().item()) // 2}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=1, help="0: skip the oracle's cpu_baseline leg")
    ap.add_argument("--kernel", default=None, choices=[None, "lb", "surrogate", "fem", "bridges", "full", "batch"],
                    help="time one kernel alone")
    ap.add_argument("--grid", default="256x128x128", help="grid of --kernel lb")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"], help="lattice storage of --kernel lb")
    ap.add_argument("--shape", type=int, default=None, help="launch shape of --kernel lb (lb_set_shape)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 16-bit storage and surrogate forms")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary configurations (FEM bending, platelet pair, batched, surrogate, "
                         "the full-scale forms)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.kernel == "lb":
        run_lb_only(args)
        return
    if args.kernel == "surrogate":
        run_surrogate_only(args)
        return
    if args.kernel == "fem":
        run_fem_only(args)
        return
    if args.kernel == "bridges":
        run_bridges_only(args)
        return
    if args.kernel == "full":
        run_full_only(args)
        return
    if args.kernel == "batch":
        run_batched_only(args)
        return
    rank, ws = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_native(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
