"""Benchmark of the coupled LB / rigid-ellipsoid time step on GB300.

Workload (default): the 128^3 shear cell of the paper's microvessel setting,
walls at z moving at -/+0.02, 1022 oblate (7,7,3) cells at 30 % volume
fraction, tau = 1, FP32 shifted population storage.  One "step" is one
coupled time step (lattice sweep with bounce-back, momentum exchange and
contact links; cell list; pair and wall potentials; leap-frog; first-arrival
re-discretisation with fill/drain).

Metric: coupled MLUPS = lattice sites x steps / time / 1e6 over all sites
(the paper's cost measure), plus the achieved fraction of the HBM roofline of
the lattice sweep (algorithmic bytes per launch / its CUDA-event duration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (launched by torchrun) every rank steps its own replica of the
workload (the single-domain path does not shard); value sums all ranks'
site updates over the slowest rank's time.  --impl reference times the FP64
CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS & % HBM roofline, plain FP32 vs BF16/FP16 store at stated error"
UNIT = "MLUPS"


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return ws, rank, local


def _cuda():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clocks, their maximum, power and the clock-event (throttle) reasons
    of the benchmarked GPU, polled every ~1 ms through NVML (the driver's
    management library, loaded with ctypes) while the timed region runs;
    nvidia-smi at its shortest interval where NVML cannot be loaded.  The GPU
    is found by its PCI bus id, so the sample is of the device the bench runs
    on even when NVML numbers the machine's GPUs differently."""

    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.samples = []  # (sm_mhz, sm_max_mhz, power_w, reasons)
        self.stop_ev = threading.Event()
        self.thread = None
        self.proc = None
        self.source = None

    def _bus_id(self):
        try:
            import torch

            pr = torch.cuda.get_device_properties(self.cuda_index)
            return "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            return None

    def _nvml(self):
        import ctypes

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        bus = self._bus_id()
        ok = bus is not None and lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, ctypes.byref(h)) != 0:
            return None
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons_fn

    def _poll_nvml(self, lib, h, reasons_fn):
        import ctypes

        mhz, mx, mw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # 1 = NVML_CLOCK_SM
        while not self.stop_ev.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0:
                pw = mw.value / 1000.0 if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(mw)) == 0 else None
                rr = rs.value if reasons_fn(h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(mhz.value), float(mx.value), pw,
                                     [n for bit, n in self.REASONS.items() if rr & bit]))
            time.sleep(0.001)

    def start(self):
        try:
            nv = self._nvml()
        except Exception:
            nv = None
        if nv is not None:
            self.source = "nvml, ~1 ms"
            self.thread = threading.Thread(target=self._poll_nvml, args=nv, daemon=True)
            self.thread.start()
            return
        try:
            bus = self._bus_id()
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", bus or str(self.cuda_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 10 ms"
            self.thread = threading.Thread(target=self._read_smi, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read_smi(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                pw = float(parts[2]) if parts[2] not in ("", "[N/A]") else None
                self.samples.append((float(parts[0]), float(parts[1]), pw,
                                     [n for n, v in zip(names, parts[3:7]) if v.lower().startswith("active")]))
            except ValueError:
                continue

    def stop(self):
        self.stop_ev.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        if self.source is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no NVML and no nvidia-smi"], "samples": 0}
        sm = [x[0] for x in self.samples]
        pw = [x[2] for x in self.samples if x[2] is not None]
        reasons = sorted({r for x in self.samples for r in x[3]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(x[1] for x in self.samples) if sm else None,
                "power_w_max": round(max(pw), 1) if pw else None,
                "reasons": reasons, "samples": len(sm), "source": self.source}


def make_workload(name):
    from paper_1005_2594_gb300 import workloads

    if name == "shear128":
        p, X, q = workloads.shear_cell(n=128, phi=0.30, U=0.02, seed=1002)
        return p, X, q, None, "shear cell 128^3, walls z +-0.02, 1022 (7,7,3) cells at 30 %"
    if name == "small32":
        p, X, q = workloads.small_shear()
        return p, X, q, None, "shear cell 32^3, walls z +-0.01, 20 (3.5,3.5,1.5) cells"
    if name == "ensemble64":  # (the reference arm samples the first member)
        p, X, q, d = workloads.ensemble(n_boxes=1, seed=1004)[0]
        return p, X, q, None, "ensemble member 0: " + d
    if name == "tube512":
        p, X, q, mask = workloads.tube()
        return p, X, q, mask, "tube 512x256x256, radius 120 along x, g = 1e-6 on plasma and cells, %d (7,7,3) cells at 35 %% of the lumen" % len(X)
    if name == "tube_rheology":
        from paper_1005_2594_gb300 import rheology

        p, X, q, mask = rheology.tube_case(1)
        return p, X, q, mask, "tube radius 30, length 128, %d (7,7,3) cells at 35 %% of the lumen, g = 2e-6" % len(X)
    if name == "vessel_loop":
        # (the reference arm's sample: the same loop at a quarter of the size)
        mask, _ = workloads.vessel_loop(256, 128, 32, 8.0, 32.0)
        p = workloads.base_params(256, 128, 32, periodic=(1, 1, 1), g=(1e-6, 0.0, 0.0))
        return p, np.zeros((0, 3)), np.zeros((0, 4)), mask, "vessel loop 256x128x32 (parent radius 8), plasma"
    if name == "le_shear":
        from paper_1005_2594_gb300 import rheology

        p, X, q = rheology.le_shear_case()
        p["le_U"] = LE_U
        return p, X, q, None, "Lees-Edwards shear cell 128x40x40, offset %g, %d (5.5,5.5,1.83) cells at 56 %%" % (
            LE_U, len(X))
    if name == "arteriole":
        from paper_1005_2594_gb300 import rheology

        p, X, q, mask = rheology.arteriole_case()
        return p, X, q, mask, "arteriole radius 46.5, length 64, %d (5.5,5.5,1.83) cells at 42 %% of the lumen, g = 8e-6" % len(X)
    if name == "duct256":
        p, X, q = workloads.duct(n=256, n_cells=8192, g=1e-6, seed=1003)
        return p, X, q, None, "duct 256^3, walls y z, g = 1e-6 along x, 8192 (7,7,3) cells"
    raise ValueError(name)


# DRAM traffic of one lattice sweep (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of the even and odd launch) from the ncu capture of the shear-cell
# workload at FP32 storage kept with the profiles, valid for the sweep source
# it was taken on (lb_sweep.cuh, first 16 hex digits of its SHA-256) and that
# workload only
SWEEP_TRAFFIC = {"sha": "bc31081e20bd634a", "config": "shear128", "store": 0, "bytes": 328095360}


SWEEP_KERNELS = {
    0: "k_lb_step (fused collide/stream/bounce-back, one node per thread, %s store)",
    1: "k_lb_step_pipe (fused collide/stream/bounce-back, per-thread copy pipeline over 4 planes, %s store)",
    2: "k_lb_step_pipe (fused collide/stream/bounce-back, per-thread copy pipeline over 8 planes, %s store)",
    3: "k_lb_step_bulk (fused collide/stream/bounce-back, bulk-copy pipeline over 8 planes, %s store)",
    4: "k_lb_step_bulk (fused collide/stream/bounce-back, bulk-copy pipeline over 4 planes, %s store)",
    5: "k_lb_step_rows (fused collide/stream/bounce-back, persistent bulk-copy row pipeline, %s store)",
}


def sweep_kernel(nx, store, variant=None, cells=True):
    """the sweep kernel the library runs for this row length, storage type
    and variant (None: the context's own choice, one node per thread with
    cells, else the bulk-copy pipeline where rows are 16-byte aligned); the
    bulk-copy variants need 16-byte aligned rows and the per-thread pipeline
    FP32, else the library runs one node per thread"""
    name = {0: "FP32", 1: "BF16", 2: "FP16"}[store]
    aligned = nx % (4 if store == 0 else 8) == 0
    if variant is None:
        variant = 0 if cells else (3 if aligned else (1 if store == 0 else 0))
    if (variant in (3, 4, 5) and not aligned) or (variant in (1, 2) and store != 0):
        variant = 0
    return SWEEP_KERNELS[variant] % name


def sweep_traffic(config, store):
    import hashlib

    src = os.path.join(ROOT, "paper_1005_2594_gb300", "csrc", "lb_sweep.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    t = SWEEP_TRAFFIC
    if sha == t["sha"] and config == t["config"] and store == t["store"]:
        return t["bytes"]
    return None


def job_value(ws, N, steps, ms_max):
    """whole-job MLUPS: every rank steps its own replica of N sites; the
    slowest rank's time counts"""
    return ws * N * steps / (ms_max * 1e-3) / 1e6


def sweep_bytes(sim, dtype_size):
    """algorithmic bytes of one lattice sweep: every fluid node reads and
    writes its 19 populations, every node's owner id is read once"""
    owner = sim.owner()
    n_fluid = int((owner == -1).sum())
    return n_fluid * 2 * 19 * dtype_size + owner.size * 4, n_fluid


def run_gpu(args, ws, rank, local):
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl

    __graft_entry__.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    p, X, q, mask, desc = make_workload(args.config)
    N = p["nx"] * p["ny"] * p["nz"]
    dsize = {0: 4, 1: 2, 2: 2}[args.store]
    sim = bl.Simulation(p, store_dtype=args.store, stream=stream.cuda_stream, wall_mask=mask)
    if args.sweep is not None:
        sim.sweep_variant(args.sweep)
    sim.set_particles(X, q)
    sim.step(args.warmup)
    sim.sync()
    launches0 = bl.bl_launch_count(sim.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    sim.sync()
    launches = bl.bl_launch_count(sim.ctx) - launches0
    # per-kernel times from a separate instrumented run (CUDA events around
    # every kernel group on the stream it runs on; no graph replay there)
    bl.bl_timing_enable(sim.ctx, True)
    bl.bl_timing_read(sim.ctx)  # clear
    k_inst = max(20, min(args.steps, 200))
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(k_inst)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_inst = e0.elapsed_time(e1)
    sim.sync()
    groups = bl.bl_timing_read(sim.ctx)
    bl.bl_timing_enable(sim.ctx, False)
    ms_max = allreduce_max(ms, ws)
    value = job_value(ws, N, args.steps, ms_max)
    k1_ms, k1_n = groups["lattice_sweep"]
    bytes_per, n_fluid = sweep_bytes(sim, dsize)
    hbm, src = peaks()
    achieved = bytes_per / (k1_ms / k1_n * 1e-3) / 1e9 if k1_n else None
    group_share = {g: round(v[0] / max(sum(x[0] for x in groups.values()), 1e-30), 4) for g, v in groups.items()}
    # end-to-end through the C ABI with host buffers: each step uploads the
    # cell state (bl_particles_set), steps once and reads back forces and state
    e2e = run_e2e(sim, X.shape[0], N, args.e2e_steps, stream)
    prec = precision_error(p, X, q, mask, args.store, args.precision_steps, stream) \
        if args.store != 0 and args.precision_steps > 0 else None
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {0: "f32", 1: "bf16", 2: "f16"}[args.store],
        "data": "synthetic (seeded random packing, resting start)",
        "config": {"workload": desc, "lattice": [p["nx"], p["ny"], p["nz"]], "cells": int(X.shape[0]),
                   "fluid_nodes": n_fluid, "store": {0: "f32", 1: "bf16", 2: "f16"}[args.store],
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "populations %.0f MB > 129 MB L2, no flush" % (N * 19 * dsize / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4) if achieved else None,
                     "traffic": sweep_traffic(args.config, args.store), "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
                     else "fallback 6.8 TB/s", "kernel": sweep_kernel(p["nx"], args.store, args.sweep),
                     "bytes_per_launch": bytes_per, "launch_ms": round(k1_ms / max(k1_n, 1), 5),
                     # the coupled step as a whole: the same algorithmic bytes (the
                     # link, contact, potential and fill/drain work adds none when
                     # fused) over the graph-replayed step time
                     "step_achieved": round(bytes_per / (ms_max / args.steps * 1e-3) / 1e9, 1),
                     "step_frac": round(bytes_per / (ms_max / args.steps * 1e-3) / 1e9 / hbm, 4)},
        "kernel_time_share": group_share,
        "instrumented": {"steps": k_inst, "ms_per_step": round(ms_inst / k_inst, 5),
                         "note": "per-kernel CUDA events, no graph replay, the sweep timed alone (the side "
                                 "streams start when it ends); roofline and shares from this run"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if prec is not None:
        out["precision_error"] = prec
    return out, (p, X, q, desc)


def run_ensemble(args, ws, rank, local):
    """64 uneven shear cells (cubes of 48..96, hematocrit 10..45 %, wall
    speeds 0.005..0.05): aggregate MLUPS of the ensemble graph against the
    same members stepped one after another, after each member's sweep
    variant is chosen by the autotuner."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    __graft_entry__.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    boxes = workloads.ensemble(n_boxes=64, seed=1004)
    sims = []
    for p, X, q, _ in boxes:
        s = bl.Simulation(p, stream=stream.cuda_stream)
        s.set_particles(X, q)
        sims.append(s)
    sites = sum(s.N for s in sims)
    choices = [s.autotune(8) for s in sims]
    ens = bl.Ensemble(sims, stream=stream.cuda_stream)
    ens.step(args.warmup)
    ens.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the members one after another (each replays its own two-step graph)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in sims:
        s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1)
    ens.sync()
    # the ensemble graph
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    ens.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ens.sync()
    ms_max = allreduce_max(ms, ws)
    fluid = sum(int((s.owner() == -1).sum()) for s in sims)
    bytes_step = fluid * 2 * 19 * 4 + sites * 4
    hbm, src = peaks()
    achieved = bytes_step * args.steps / (ms_max * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(job_value(ws, sites, args.steps, ms_max), 2), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded random packings, resting start)",
        "config": {"workload": "ensemble of 64 shear cells, cubes 48..96, hematocrit 10..45 %, U 0.005..0.05",
                   "members": len(sims), "sites": sites, "cells": int(sum(len(b[1]) for b in boxes)),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "populations %.0f MB > 129 MB L2, no flush" % (sites * 19 * 4 / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None,
                     "kernel": "whole ensemble step (sweep bytes over step time)",
                     "peak_source": src},
        "serial": {"value": round(sites * args.steps / (ms_serial * 1e-3) / 1e6, 2),
                   "ms_per_step": round(ms_serial / args.steps, 5),
                   "note": "the same members stepped one after another on one stream"},
        "autotune": {str(v): choices.count(v) for v in sorted(set(choices))},
        "clocks": clk,
    }
    ens.close()
    return out


def run_learned(args, ws, rank, local):
    """The learned near-contact correction: the network is trained through
    the library on approach runs it generates (coarse and 2x resolution),
    its error is measured on held-out approach runs against the 2x and 4x
    runs, and the tube workload is timed without and with the network
    attached for pairs from the smallest trained gap up to 2 lattice units
    (closer pairs keep the plain method)."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import learned

    __graft_entry__.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    X, Y, _, runs = learned.approach_samples(64, seed=11)
    Xh, Yh, _, _ = learned.approach_samples(20, seed=12)
    X4, Y4, _, _ = learned.approach_samples(8, seed=13, k=4)
    t_data = time.time() - t0
    t0 = time.time()
    m, info = learned.fit(X, Y, runs, seed=0)
    torch.cuda.synchronize()
    t_fit = time.time() - t0
    scale = Y.std(axis=0)
    e2 = learned.errors(m, Xh, Yh, scale)
    e4 = learned.errors(m, X4, Y4, scale)
    P = learned.predict(m, Xh)

    def rms_ratio(a, b):
        return float(np.sqrt(((Yh - P)[:, a:b] ** 2).sum(1).mean() / (Yh[:, a:b] ** 2).sum(1).mean()))

    p, Xc, qc, mask, desc = make_workload("tube512")
    N = p["nx"] * p["ny"] * p["nz"]
    sim = bl.Simulation(p, stream=stream.cuda_stream, wall_mask=mask)
    sim.set_particles(Xc, qc)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    clocks = ClockSampler(local)
    for mode in ("plain", "learned"):
        if mode == "learned":
            # the trained gaps from below, up to the cut-off; closer pairs keep the plain method
            bl.bl_mlp_attach_range(sim.ctx, m, info["gap_min"], 2.0, info["speed_min"], info["speed_max"])
        sim.step(args.warmup)
        sim.sync()
        l0 = bl.bl_launch_count(sim.ctx)
        if mode == "learned":
            clocks.start()
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ms = allreduce_max(e0.elapsed_time(e1), ws)
        sim.sync()
        res[mode] = (ms, bl.bl_launch_count(sim.ctx) - l0)
    clk = clocks.stop()
    ms, launches = res["learned"]
    ms_plain = res["plain"][0]
    fluid = int((sim.owner() == -1).sum())
    hbm, src = peaks()
    bytes_step = fluid * 2 * 19 * 4 + N * 4
    achieved = bytes_step * args.steps / (ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(job_value(ws, N, args.steps, ms), 2), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network bf16)",
        "data": "synthetic (jittered fcc start, resting plasma; network trained on generated approach runs)",
        "config": {"workload": desc, "lattice": [p["nx"], p["ny"], p["nz"]], "cells": int(len(Xc)),
                   "fluid_nodes": fluid, "gap_range": [round(info["gap_min"], 3), 2.0],
                   "speed_range": [round(info["speed_min"], 4), round(info["speed_max"], 4)], "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "populations %.0f MB > 129 MB L2, no flush" % (N * 19 * 4 / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None,
                     "kernel": "whole coupled step with the network (sweep bytes over step time)", "peak_source": src},
        "without_network": {"value": round(job_value(ws, N, args.steps, ms_plain), 2),
                            "ms_per_step": round(ms_plain / args.steps, 5)},
        "learned": {
            "approach_runs": {"train": 64, "held_out_2x": 20, "held_out_4x": 8, "generation_s": round(t_data, 1)},
            "training": {"seconds": round(t_fit, 2), **{k: (round(v, 4) if isinstance(v, float) else v)
                                                         for k, v in info.items()}},
            "error_vs_2x": {"without": round(e2[0], 4), "with": round(e2[1], 4), "ratio": round(e2[1] / e2[0], 4),
                            "force_rms_ratio": round(rms_ratio(0, 3), 4),
                            "torque_rms_ratio": round(rms_ratio(3, 6), 4)},
            "error_vs_4x": {"without": round(e4[0], 4), "with": round(e4[1], 4), "ratio": round(e4[1] / e4[0], 4)},
            "note": "mean squared error of the body-frame hydrodynamic force and torque on held-out approach "
                    "runs, each output divided by its spread in the training data"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    sim.close()
    bl.bl_mlp_destroy(m)
    return out


def precision_error(p, X, q, mask, store, steps, stream):
    """Reduced-precision storage against FP32 storage (which matches the FP64
    oracle to 1e-5 over 100 steps at 32^3): both from the same state, `steps`
    steps.  Over that many steps a cell can cross a node a step earlier in one
    run than in the other; the node is then refilled at another time and its
    velocity differs by the cell's, so besides the RMS error over the common
    fluid nodes the largest error is given over the nodes at least 3 nodes
    away from any owner difference, with the number of owner differences;
    cell positions: the largest difference in lattice units."""
    import numpy as np
    from scipy import ndimage

    from paper_1005_2594_gb300 import bloodlb as bl

    out = []
    for st in (0, store):
        sim = bl.Simulation(p, store_dtype=st, stream=stream.cuda_stream, wall_mask=mask)
        sim.set_particles(X, q)
        sim.step(steps)
        sim.sync()
        _, u, own = sim.fields()
        out.append((u, own, sim.particles()["X"]))
        sim.close()
    (u0, o0, X0), (u1, o1, X1) = out
    fl = (o0 == -1) & (o1 == -1)
    diff = (o0 != o1).reshape(p["nz"], p["ny"], p["nx"])
    near = ndimage.binary_dilation(diff, structure=np.ones((3, 3, 3), bool), iterations=3,
                                   border_value=0).reshape(-1)
    away = fl & ~near
    e = np.linalg.norm(u1 - u0, axis=1)
    scale = np.abs(u0[fl]).max()
    d = X1 - X0
    for k, n in enumerate((p["nx"], p["ny"], p["nz"])):
        d[:, k] -= n * np.round(d[:, k] / n)
    return {"vs": "FP32 storage", "steps": steps,
            "u_rel_rms": float(np.sqrt((e[fl] ** 2).mean() / (np.linalg.norm(u0[fl], axis=1) ** 2).mean())),
            "u_rel_max_away": float(e[away].max() / scale) if away.any() else None,
            "u_rel_max": float(e[fl].max() / scale),
            "owner_differences": int(diff.sum()), "X_max_abs": float(np.abs(d).max())}


def run_rheology(args, ws, rank, local):
    """Apparent viscosity (relative to the plasma) of a tube suspension: a
    tube of radius 30 and length 128 with (7,7,3) cells at 35 % of the lumen,
    driven by g = 2e-6 on plasma and cells, from rest: the coarse method
    alone, with the learned correction (trained here on approach runs), and
    the plain method at 2x resolution (4x the steps); each against the
    plasma alone at its resolution.  Coarse runs take --steps steps (about
    20000 reach steady flow), the 2x runs four times as many."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import learned, rheology

    __graft_entry__.build()
    torch.cuda.set_device(local)
    X, Y, _, runs = learned.approach_samples(64, seed=11)
    m, info = learned.fit(X, Y, runs, seed=0)
    rng = (info["gap_min"], 2.0, info["speed_min"], info["speed_max"])
    res, profiles = {}, {}
    for name, k, cells, net in (("plasma_1x", 1, False, False), ("plain_1x", 1, True, False),
                                ("learned_1x", 1, True, True), ("plasma_2x", 2, False, False),
                                ("plain_2x", 2, True, False)):
        p, Xc, qc, mask = rheology.tube_case(k, cells=cells)
        steps = args.steps * k * k
        Q, samples, ms, prof = rheology.run(p, Xc, qc, mask, steps, model=m if net else None, gap_range=rng,
                                            profile_radius=30.0 * k)
        N = p["nx"] * p["ny"] * p["nz"]
        res[name] = {"flux": Q, "flux_rel_spread": float(np.std(samples) / abs(Q)), "steps": steps,
                     "cells": int(len(Xc)), "lattice": [p["nx"], p["ny"], p["nz"]],
                     "mlups": N * steps / (ms * 1e-3) / 1e6}
        profiles[name] = prof
    mu = {"plain_1x": res["plasma_1x"]["flux"] / res["plain_1x"]["flux"],
          "learned_1x": res["plasma_1x"]["flux"] / res["learned_1x"]["flux"],
          "plain_2x": res["plasma_2x"]["flux"] / res["plain_2x"]["flux"]}
    # Sec. IV: the plasma-only profile places the staircase wall (its
    # effective radius); each suspension's profile is then fitted with the
    # two-layer model, the boundary viscosity set to the plasma's
    # (lengths in coarse lattice units; the 2x lattice's force density is
    # g / 8 in its own units)
    mu_b = p["rho0"] * (p["tau"] - 0.5) / 3.0
    fits = {}
    for k, plasma, susp in ((1, "plasma_1x", ("plain_1x", "learned_1x")), (2, "plasma_2x", ("plain_2x",))):
        f = p["rho0"] * 2e-6 / k ** 3
        r_c, u_p, _, n_p = profiles[plasma]
        R_eff = rheology.fit_poiseuille_radius(r_c, u_p, f, mu_b, n_p)
        fits["R_eff_%dx" % k] = round(R_eff / k, 4)
        for name in susp:
            r_s, u_s, H, n_s = profiles[name]
            d, mr = rheology.fit_axial_train(r_s, u_s, R_eff, f, mu_b, n_s)
            Rc = R_eff - d
            fits[name] = {"delta": round(d / k, 4), "mu_c_over_mu_b": round(mr, 4),
                          "mu_rel_of_fit": round(R_eff ** 4 / (R_eff ** 4 - Rc ** 4 + Rc ** 4 / mr), 4)}
            if k == 1:
                fits[name].update({"u_axial": [round(float(v), 9) for v in u_s],
                                   "H": [round(float(v), 4) for v in H]})
        if k == 1:
            fits["r"] = [float(v) for v in r_c]
            fits["u_axial_plasma"] = [round(float(v), 9) for v in u_p]
    r = res["learned_1x"]
    out = {
        "metric": METRIC, "value": round(r["mlups"], 2), "unit": UNIT, "n_gpus": ws, "steps": r["steps"],
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (network bf16)", "data": "synthetic (jittered fcc start, resting plasma)",
        "config": {"workload": "tube radius 30, length 128, %d (7,7,3) cells at 35 %% of the lumen, g = 2e-6; "
                               "value: coarse with the network (MLUPS of the stepping)" % r["cells"],
                   "lattice": r["lattice"], "gap_range": [round(rng[0], 3), rng[1]],
                   "speed_range": [round(rng[2], 4), round(rng[3], 4)]},
        "rheology": {"mu_rel": {k: round(v, 4) for k, v in mu.items()},
                     "note": "apparent viscosity relative to the plasma = plasma flux / suspension flux under the "
                             "same driving, flux averaged over the second half of each run from rest",
                     "runs": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                              for k, v in res.items()},
                     "profiles": fits,
                     "profiles_note": "radial bins of unit width about the tube axis, averaged over the flux samples: "
                                      "mean axial velocity of the fluid nodes and cell fraction H; R_eff from the "
                                      "plasma-only profile, delta and mu_c/mu_b from the two-layer fit of the "
                                      "suspension's profile (boundary viscosity = plasma's, f = rho g)"},
        "roofline": None,
    }
    bl.bl_mlp_destroy(m)
    return out


def run_arteriole(args, ws, rank, local):
    """Sec. IV's arteriole (radius 31 um = 46.5 nodes, periodic length 64,
    cells sigma = (6, 2), R = 11/12 sigma, 42 % of the lumen, cell-wall
    stiffness 1.47e-16 J) driven from rest for --steps steps (60000 let the
    fcc start dissolve): the radial velocity profile fitted with the two-layer
    model (cell-depleted layer width delta, core-to-boundary viscosity ratio)
    and the cell fraction H(r), with the wall radius taken from the plasma
    alone under the same force.  Two fcc starts: centres kept R_perp + 1
    from the wall (no cell reaches it) and R_par + 1 (edge-on cells reach
    into it); the second also at 10 and 100 times and a tenth of the
    cell-wall stiffness, the paper's knob for the layer width.  A run that the
    library stops as unstable is reported as such."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import rheology

    __graft_entry__.build()
    torch.cuda.set_device(local)
    g = 8e-6
    p, _, _, mask = rheology.arteriole_case(cells=False, g=g)
    f, mu_b = p["rho0"] * g, p["rho0"] * (p["tau"] - 0.5) / 3.0
    Qp, _, msp, (r_c, u_p, _, n_p) = rheology.run(p, np.zeros((0, 3)), np.zeros((0, 4)), mask, args.steps,
                                                   profile_radius=31.0 / rheology.DX_UM)
    R_eff = rheology.fit_poiseuille_radius(r_c, u_p, f, mu_b, n_p)
    runs = {}
    for name, ew, start in (("wide start, eps_w 1.47e-16 J", 1.47e-16, "wide"),
                            ("close start, eps_w 1.47e-16 J", 1.47e-16, "close"),
                            ("close start, eps_w 1.47e-15 J", 1.47e-15, "close"),
                            ("close start, eps_w 1.47e-14 J", 1.47e-14, "close"),
                            ("close start, eps_w 1.47e-17 J", 1.47e-17, "close")):
        p, X, q, mask = rheology.arteriole_case(g=g, eps_w_J=ew, start=start)
        try:
            Q, samples, ms, (r_c, u_s, H, n_s) = rheology.run(p, X, q, mask, args.steps,
                                                              profile_radius=31.0 / rheology.DX_UM)
        except bl.BloodLBError as e:  # the library's stability check (a host-read status)
            runs[name] = {"eps_w": round(p["eps_w"], 6), "cells": int(len(X)), "failed": str(e)}
            continue
        d, mr = rheology.fit_axial_train(r_c, u_s, R_eff, f, mu_b, n_s)
        Rc = R_eff - d
        N = p["nx"] * p["ny"] * p["nz"]
        runs[name] = {"eps_w": round(p["eps_w"], 6), "cells": int(len(X)), "flux": round(Q, 5),
                      "flux_rel_spread": round(float(np.std(samples) / abs(Q)), 5),
                      "pseudo_shear_rate_per_s": round(rheology.pseudo_shear_rate(Q, R_eff), 1),
                      "mu_rel": round(Qp / Q, 4), "delta_nodes": round(d, 3),
                      "delta_um": round(d * rheology.DX_UM, 3), "mu_c_over_mu_b": round(mr, 3),
                      "mu_rel_of_fit": round(R_eff ** 4 / (R_eff ** 4 - Rc ** 4 + Rc ** 4 / mr), 4),
                      "H_axis": round(float(np.nanmean(H[:5])), 4),
                      "mlups": round(N * args.steps / (ms * 1e-3) / 1e6, 1),
                      "u_axial": [round(float(v), 9) for v in u_s], "H": [round(float(v), 4) for v in H]}
    main = runs["close start, eps_w 1.47e-16 J"]
    return {
        "metric": METRIC, "value": main["mlups"], "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (jittered fcc start, resting plasma)",
        "config": {"workload": "arteriole radius 31 um (46.5 nodes), periodic length 64, %d cells sigma (6,2) "
                               "R = 11/12 sigma at 42 %% of the lumen, g = %g on plasma and cells; value: MLUPS "
                               "of the stepping at the paper's cell-wall stiffness" % (main["cells"], g), "g": g,
                   "lattice": [p["nx"], p["ny"], p["nz"]]},
        "arteriole": {"R_eff_nodes": round(R_eff, 4), "plasma_flux": round(Qp, 5),
                      "paper": {"mu_c_over_mu_b": "2.43 +- 0.01", "delta_um": "1.47 +- 0.04",
                                "pseudo_shear_rate_per_s": 1.3e3, "H_axis": "up to about 0.6"},
                      "r_nodes": [float(v) for v in r_c], "u_axial_plasma": [round(float(v), 9) for v in u_p],
                      "runs": runs,
                      "note": "radial bins of unit width about the axis, averaged over 20 samples in the second "
                              "half; two-layer fit with the boundary viscosity the plasma's and the wall radius "
                              "fitted to the plasma alone; mu_rel = plasma flux / suspension flux"},
        "roofline": None,
    }


# Lees-Edwards offset of the shear cell: Sec. IV's shear rate 2.21e3 / s is
# 1.50e-4 per step (dt = 6.80e-8 s), times l_x = 128
LE_U = 0.0192


def run_le_shear(args, ws, rank, local):
    """Sec. IV's apparent viscosity in plane Couette flow (Eq. mu): the shear
    cell 128 x 40 x 40 under the Lees-Edwards offset LE_U, from rest for
    --steps steps (60000: a strain of about 9), plasma alone (mu_rel must be
    1) and the suspension of 388 cells at the paper's 56 %; Delta p_LE and the
    shear rate (linear fit over the central half) averaged over the second
    half.  value: MLUPS of the suspension's stepping."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import rheology

    __graft_entry__.build()
    torch.cuda.set_device(local)
    runs = {}
    for name, cells in (("plasma", False), ("suspension", True)):
        p, X, q = rheology.le_shear_case(cells=cells)
        r = rheology.run_le(p, X, q, LE_U, args.steps)
        N = p["nx"] * p["ny"] * p["nz"]
        runs[name] = {"cells": int(len(X)), "mu_rel": round(r["mu_rel"], 4),
                      "gamma_dot_per_step": r["gamma_dot"], "gamma_dot_per_s": round(r["gamma_dot_per_s"], 1),
                      "P_per_step": r["P_per_step"], "mlups": round(N * args.steps / (r["ms"] * 1e-3) / 1e6, 1),
                      "profile": [round(float(v), 7) for v in r["profile"]]}
    s = runs["suspension"]
    return {
        "metric": METRIC, "value": s["mlups"], "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (jittered fcc start, resting plasma)",
        "config": {"workload": "Lees-Edwards shear cell 128x40x40, offset %g, %d cells sigma (6,2) R = 11/12 sigma "
                               "at the paper's 6.4e15 / m^3 (56 %%); value: MLUPS of the suspension's stepping"
                               % (LE_U, s["cells"]), "U": LE_U},
        "lees_edwards": {"runs": runs,
                         "paper": {"gamma_dot_per_s": "2.21e3 +- 0.08e3"},
                         "note": "mu_rel = -<Delta p_LE> / (l_y l_z gamma_dot mu), Eq. (mu), over the second half; "
                                 "gamma_dot from a linear fit of v_z(x) over the central half"},
        "roofline": None,
    }


def run_vessel_loop(args, ws, rank, local):
    """The indexed lattice (only fluid nodes stored and swept) against the
    dense lattice on one sparse geometry: the synthetic vessel loop
    1024 x 512 x 128, parent radius 32 splitting into two daughters of radius
    25.4 that rejoin (6.1 % of the box is lumen), plasma driven by g = 1e-6
    along x.  Each path takes --warmup untimed and --steps timed steps (graph
    replays), timed with CUDA events; throughput counts fluid nodes.  The
    roofline is the indexed sweep's: per fluid node 2 x 19 populations plus
    the 18 neighbour indices."""
    import torch

    import __graft_entry__
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    __graft_entry__.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    nx, ny, nz = 1024, 512, 128
    mask, _ = workloads.vessel_loop(nx, ny, nz, 32.0, 128.0)
    p = workloads.base_params(nx, ny, nz, periodic=(1, 1, 1), g=(1e-6, 0.0, 0.0))
    N = nx * ny * nz
    dsize = {0: 4, 1: 2, 2: 2}[args.store]

    def timed(obj, launch_count):
        obj.step(args.warmup)
        obj.sync()
        l0 = launch_count()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        obj.sync()
        return e0.elapsed_time(e1), launch_count() - l0

    sp = bl.SparseLattice(p, wall_mask=mask, store_dtype=args.store, stream=stream.cuda_stream)
    nf = sp.n_fluid
    clocks = ClockSampler(local)
    clocks.start()
    ms_sp, launches = timed(sp, sp.launch_count)
    clk = clocks.stop()
    _, u_sp = sp.fields()
    sp.close()
    dn = bl.Simulation(p, store_dtype=args.store, stream=stream.cuda_stream, wall_mask=mask)
    ms_dn, _ = timed(dn, lambda: bl.bl_launch_count(dn.ctx))
    _, u_dn, _ = dn.fields()
    dn.close()
    fl = mask == 0
    diff = float(np.abs(u_sp[fl] - u_dn[fl]).max() / max(np.abs(u_dn[fl]).max(), 1e-30))
    hbm, src = peaks()
    bytes_per_node = 2 * 19 * dsize + 18 * 4
    achieved = bytes_per_node * nf / (ms_sp / args.steps * 1e-3) / 1e9
    value = nf * args.steps / (ms_sp * 1e-3) / 1e6
    mem_sp = nf * (19 * dsize + 18 * 4 + 4)
    mem_dn = N * (19 * dsize + 4 + 4 + 4 + 16)
    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT + " (fluid nodes)", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_sp / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "bf16", 2: "f16"}[args.store], "data": "synthetic (vessel loop geometry, plasma)",
        "config": {"workload": "vessel loop 1024x512x128 (parent radius 32, daughters 25.4), indexed lattice, "
                               "g = 1e-6; value: fluid-node updates per second",
                   "fluid_nodes": int(nf), "box_nodes": int(N), "lumen_fraction": round(nf / N, 4),
                   "l2": "indexed populations and table %.0f MB > 129 MB L2, no flush" % (mem_sp / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None,
                     "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6.8 TB/s",
                     "kernel": "k_sparse_step (indexed AA sweep, one fluid node per thread)",
                     "bytes_per_launch": bytes_per_node * nf, "launch_ms": round(ms_sp / args.steps, 5)},
        "dense_lattice": {"ms_per_step": round(ms_dn / args.steps, 5),
                          "mlups_fluid_nodes": round(nf * args.steps / (ms_dn * 1e-3) / 1e6, 1),
                          "mlups_box_nodes": round(N * args.steps / (ms_dn * 1e-3) / 1e6, 1),
                          "speedup_of_indexed": round(ms_dn / ms_sp, 2),
                          "u_rel_diff_vs_indexed": diff},
        "memory_bytes": {"indexed": int(mem_sp), "dense": int(mem_dn), "ratio": round(mem_dn / mem_sp, 1)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }


def run_e2e(sim, n, N, steps, stream):
    import torch

    from paper_1005_2594_gb300 import bloodlb as bl

    if steps <= 0:
        return None
    st = sim.particles()
    Xh, qh, Vh, Lh = (np.ascontiguousarray(st[k]) for k in ("X", "q", "V", "L"))
    sim.sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.set_particles(Xh, qh, Vh, Lh)
        sim.step(1)
        st = sim.particles()
        Xh, qh, Vh, Lh = st["X"], st["q"], st["V"], st["L"]
    sim.sync()
    dt = time.perf_counter() - t0
    return {"value": round(N * steps / dt / 1e6, 2), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": n * 13 * 8, "d2h_bytes_per_step": n * 19 * 8,
            "path": "bl_particles_set(host X,q,V,L) + bl_step(1) + bl_forces_get(host F,T,X,q,V,L)"}


def cpu_oracle_step_time(p, X, q, nsteps=1):
    import oracle

    o = oracle.Oracle(p)
    o.set_particles(X, q)
    t0 = time.perf_counter()
    o.step(nsteps)
    return (time.perf_counter() - t0) / nsteps


def _oracle_worker(p, X, q, mask, warmup, steps, barrier, out):
    """one process of the all-core oracle timing: its own copy of the sample,
    stepped after every process has set up"""
    import oracle

    o = oracle.Oracle(p)
    if mask is not None:
        o.set_walls(mask)
    if "le_U" in p:  # the Lees-Edwards shear cell
        o.set_lees_edwards(p["le_U"])
    o.set_particles(X, q)
    o.step(warmup)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(steps)
    out.put(time.perf_counter() - t0)


def host_cores(sites):
    """processes for the all-core oracle timing: one per core, as many as
    60 % of the available host memory holds (the oracle keeps about 0.5 KB
    per lattice site)"""
    n = os.cpu_count() or 1
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                n = min(n, max(1, int(int(ln.split()[1]) * 1024 * 0.6 // (sites * 500))))
    except OSError:
        pass
    return n


def cpu_model():
    try:
        for ln in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_all_cores(p, X, q, mask, warmup, steps, procs=None):
    """The FP64 oracle, as it stands (single-threaded C), run as one process
    per host core, each stepping its own copy of the sample; the processes
    start stepping together (a barrier after set-up).  Returns the aggregate
    MLUPS (every process's site updates over the slowest process's time),
    the process count and the slowest time.  Processes are spawned, never
    forked, since this process has used the GPU."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    Ns = p["nx"] * p["ny"] * p["nz"]
    n = procs or host_cores(Ns)
    barrier, out = ctx.Barrier(n), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(p, X, q, mask, warmup, steps, barrier, out)) for _ in range(n)]
    for pr in ps:
        pr.start()
    times = [out.get() for _ in ps]
    for pr in ps:
        pr.join()
    return n * Ns * steps / max(times) / 1e6, n, max(times)


def reference_sample(p, X, q, budget_s, nsteps):
    """largest lateral sub-box of the workload (same height, walls, wall speed,
    cell shape and volume fraction) whose oracle steps fit the time budget"""
    from paper_1005_2594_gb300 import workloads

    full = p["nx"] * p["ny"] * p["nz"]
    # the oracle's re-discretisation visits every node for every cell, so
    # its step costs ~ N * n_cells (12 s for 128^3 with 1022 cells)
    t_full = 12.0 * (full / 128 ** 3) * (len(X) / 1022.0)
    for fx, fy in ((1, 1), (2, 1), (2, 2), (4, 2), (4, 4), (8, 4), (8, 8)):
        nx, ny = max(p["nx"] // fx, 16), max(p["ny"] // fy, 16)
        frac = nx * ny / (p["nx"] * p["ny"])
        if t_full * frac * frac * nsteps <= budget_s or (fx, fy) == (8, 8):
            break
    if (nx, ny) == (p["nx"], p["ny"]):
        return p, X, q, "the full workload"
    sp = dict(p)
    sp["nx"], sp["ny"] = nx, ny
    n = max(1, int(round(len(X) * frac)))
    sX, sq, _ = workloads.pack_cells(sp, n, 1002)
    return sp, sX, sq, "%dx%dx%d sub-box of the workload (same walls, wall speed, cells, volume fraction), %d cells" % (
        nx, ny, p["nz"], n)


def run_reference(args, ws, rank):
    """FP64 CPU oracle on the host cores, bounded sample of the same workload."""
    if rank != 0:
        return None
    p, X, q, _mask, desc = make_workload(args.config)
    steps, warmup = args.steps, args.warmup
    if args.config in ("tube_rheology", "arteriole", "le_shear", "vessel_loop"):
        # the whole lattice (seconds per oracle step at most): as many steps as fit
        sp, sX, sq, smask = p, X, q, _mask
        steps, warmup = max(1, min(steps, 100)), min(warmup, 3)
        sample = "the whole lattice (%dx%dx%d, %d cells), %d steps" % (p["nx"], p["ny"], p["nz"], len(sX), steps)
    elif args.config == "tube512":
        # the cross-section is fixed by the radius: a slab of 8 x-planes of the
        # same tube, and as many steps as fit the budget (~0.5 s each)
        from paper_1005_2594_gb300 import workloads

        sp, sX, sq, smask = workloads.tube(nx=8)
        steps, warmup = max(1, min(steps, 200)), min(warmup, 3)
        sample = "8x256x256 slab of the same tube (walls, fcc start, 35 %% of the lumen), %d cells, %d steps" % (
            len(sX), steps)
    else:
        sp, sX, sq, sample = reference_sample(p, X, q, 150.0, steps + warmup)
        smask = None
    v, n, dt = oracle_all_cores(sp, sX, sq, smask, warmup, steps)
    unit = UNIT
    if args.config == "vessel_loop":
        # the indexed lattice counts fluid-node updates: so does its reference
        v *= float((smask == 0).mean())
        unit = UNIT + " (fluid nodes)"
    sample = "%s, one copy per process in %d processes (one per host core) stepping together" % (sample, n)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": unit, "n_gpus": ws,
            "steps": steps, "warmup": warmup, "ms_per_step": round(dt / steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random packing, resting start)",
            "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": round(v, 4), "unit": unit, "cores": n, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": round(v, 4), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--config", default="shear128", choices=["shear128", "small32", "duct256", "ensemble64", "tube512", "tube_rheology",
                                                          "arteriole", "le_shear", "vessel_loop"])
    ap.add_argument("--store", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--sweep", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="sweep variant (default: the library's choice for the row length and storage)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision-steps", type=int, default=1000,
                    help="with --store 1|2: steps of the error check against FP32 storage (0: none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.config in ("ensemble64", "tube512", "tube_rheology", "arteriole", "le_shear", "vessel_loop"):
        fn = {"ensemble64": run_ensemble, "tube512": run_learned, "tube_rheology": run_rheology,
              "arteriole": run_arteriole, "le_shear": run_le_shear, "vessel_loop": run_vessel_loop}[args.config]
        out = fn(args, ws, rank, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out, (p, X, q, desc) = run_gpu(args, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            N = p["nx"] * p["ny"] * p["nz"]
            v, n, t = oracle_all_cores(p, X, q, None, 0, 1)
            t1 = cpu_oracle_step_time(p, X, q, 1)
            out["cpu_baseline"] = {
                "value": round(v, 4), "unit": UNIT, "cores": n, "kind": "oracle",
                "sample": "1 coupled step of the same workload in each of %d processes (the single-threaded FP64 C "
                          "oracle, one process per host core, stepping together), %.1f s" % (n, t),
                "cpu": cpu_model(), "single_core": {"value": round(N / t1 / 1e6, 4), "cores": 1}}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
