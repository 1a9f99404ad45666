#!/usr/bin/env python
"""Throughput of the 6D split step: 6D cell-updates per second.

Default workload: the 32^3 x 32^3 FP32 Jeans box (1.07e9 cells, 4.3 GB),
synthetic seeded Maxwellian with one density mode, periodic, adaptive dt.  A
step is one whole split step of the hot path: half kick (3 velocity sweeps),
drift (3 position sweeps), density, FFT Poisson solve, force, dt, half kick
(the steady-state pass fuses the two half kicks of consecutive steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica on its own GPU (the path has no exchange step); value is
the sum over ranks of the cells updated divided by the slowest rank's time.
The reference arm times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "6D cell-updates/s per split step"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="jeans32_f32")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--profile-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--adjoint-steps", type=int, default=3)
    p.add_argument("--adjoint-workload", default="jeans32_modes3")
    p.add_argument("--fp64-steps", type=int, default=20)
    p.add_argument("--cpu-sample", type=float, default=1.0 / 64)
    return p.parse_args()


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------

class Ranks:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            import torch
            if torch.cuda.is_available():
                self.pg.barrier(device_ids=[self.local])
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(rank_ms: float, cells_per_rank: float, steps: int, ranks: Ranks):
    """Whole-job throughput: all ranks' cell updates over the slowest rank."""
    ms = ranks.max(rank_ms)
    return ms, ranks.world * cells_per_rank * steps / (ms / 1e3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (test infrastructure): bounded sample of one split step
# ---------------------------------------------------------------------------

def oracle_threads() -> int:
    """Threads the oracle's OpenMP loops run on."""
    from oracle import vp_oracle as O
    return O.threads()


def oracle_density(w, f0_np):
    """The oracle's density of the whole grid, slab by slab."""
    import numpy as np
    from oracle import vp_oracle as O
    grid = O.Grid.of(w)
    slab = O.Grid((1,) + tuple(w.n[1:]), grid.nv, grid.lo, grid.hi, grid.vlo, grid.vhi)
    return np.concatenate([O.density(np.ascontiguousarray(f0_np[i:i + 1], dtype=np.float64), slab)
                           for i in range(w.n[0])])


def oracle_step_rate(w, f0_np, fraction: float, rho_full=None):
    """Times the FP64 oracle on a sample of one split step of workload w and
    scales it to the whole step: the density (slab by slab: of the whole grid,
    or, given the whole density rho_full for the field solve, of the same
    fraction of x planes as the kick, scaled), the Poisson solve and force,
    the six velocity sweeps on a fraction of the velocity cubes and the three
    position sweeps on the whole lines of a fraction of the velocity cells.
    Returns (cell-updates/s, seconds per full step, description)."""
    import numpy as np
    from oracle import vp_oracle as O
    grid = O.Grid.of(w)
    nx, ny, nz = w.n
    nvx, nvy, nvz = w.nv
    sx = max(1, min(nx, int(round(fraction * nx))))
    nd = nx if rho_full is None else sx
    t0 = time.perf_counter()
    slab = O.Grid((1, ny, nz), grid.nv, grid.lo, grid.hi, grid.vlo, grid.vhi)
    rho = np.concatenate([O.density(np.ascontiguousarray(f0_np[i:i + 1], dtype=np.float64), slab)
                          for i in range(nd)])
    t_dens = (time.perf_counter() - t0) * nx / nd
    if rho_full is not None:
        rho = rho_full
    t0 = time.perf_counter()
    phi = O.poisson(rho, grid, w.G, w.poisson_bc)
    g = O.force(phi, grid, w.poisson_bc)
    dt = O.timestep(g, grid, w.courant) if w.dt_fixed <= 0 else w.dt_fixed
    t_field = time.perf_counter() - t0
    # velocity sweeps on a block of whole cubes (both half kicks)
    fk = np.ascontiguousarray(f0_np[:sx], dtype=np.float64)
    qk = fk.size / f0_np.size
    t0 = time.perf_counter()
    for _ in range(2):
        for a in range(3):
            O.sweep(fk, 3 + a, np.ascontiguousarray(g[a][:sx]), dt / 2, grid.dv[a], False)
    t_kick = time.perf_counter() - t0
    # position sweeps on the whole lines of a block of velocity cells
    svx = max(1, min(nvx, int(round(fraction * nvx))))
    fd = np.ascontiguousarray(f0_np[:, :, :, :svx], dtype=np.float64)
    qd = fd.size / f0_np.size
    t0 = time.perf_counter()
    for a in (2, 1, 0):
        O.sweep(fd, a, grid.vc(a)[:svx] if a == 0 else grid.vc(a), dt, grid.dx[a],
                w.space_bc == "periodic")
    t_drift = time.perf_counter() - t0
    full = t_dens + t_field + t_kick / qk + t_drift / qd
    dens = ("density of the whole grid" if nd == nx else
            f"density timed on {nd} of {nx} x planes and scaled")
    desc = (f"FP64 oracle, one split step of {w.name}: {dens}, the "
            f"Poisson solve timed in full; the 6 velocity sweeps timed on {sx * ny * nz} of "
            f"{nx * ny * nz} velocity cubes ({qk:.4f}) and the 3 position sweeps on the lines of "
            f"{svx * nvy * nvz} of {nvx * nvy * nvz} velocity cells ({qd:.4f}), each scaled by "
            f"its fraction; full step {full:.1f} s")
    return w.cells / full, full, desc


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

# above this many bytes of f the input is built on the device (no host copy,
# so no end-to-end and no CPU-baseline lines)
HOST_F_LIMIT = 16 << 30


def device_initial_condition(w, dev, dtype):
    """initial_condition(w) built on the device from its two FP64 factors
    (rho(x), M(v)): the same products, rounded once."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    rho, mv = I.factors(w)
    r = torch.from_numpy(rho).to(dev)
    m = torch.from_numpy(mv).to(dev)
    f = torch.empty((r.numel(), m.numel()), dtype=dtype, device=dev)
    step = max(1, (1 << 26) // m.numel())
    for s in range(0, r.numel(), step):
        f[s:s + step] = (r[s:s + step, None] * m[None, :]).to(dtype)
    return f.reshape(w.shape)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("vp_sweep.cu", "vp_sweep_fast.cu", "vp_fast_line.cuh", "vp_line.cuh", "vp_device.cuh"):
        with open(os.path.join(ROOT, "paper_1206_6152_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        ent = d[kernel]
        if ent.get("source_hash") != kernel_source_hash():
            return None
        return float(ent["dram_bytes_per_launch_full"])
    except Exception:
        return None


def run_ours(args, ranks: Ranks):
    import numpy as np
    import torch

    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of

    w = I.WORKLOADS[args.workload]()
    dev = torch.device("cuda", ranks.local)
    torch.cuda.set_device(dev)
    large = w.cells * (4 if w.dtype == "f32" else 8) > HOST_F_LIMIT and w.ic != "king"
    if large:
        # f built on the device from the two factors of the initial condition
        f0 = None
        f = device_initial_condition(w, dev, torch.float32 if w.dtype == "f32" else torch.float64)
    else:
        f0 = I.initial_condition(w)
        f = torch.from_numpy(f0).to(dev)
    stream = torch.cuda.current_stream(dev)
    sim = VlasovPoisson(config_of(w), f, stream)
    esize = f.element_size()

    # warm-up (builds the graphs)
    sim.step(max(args.warmup, 3))
    torch.cuda.synchronize(dev)

    k0 = sim.kernels_launched()
    clocks = Clocks(dev.index if dev.index is not None else 0)
    ranks.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ranks.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = sim.kernels_launched() - k0
    ms_max, value = aggregate(ms, w.cells, args.steps, ranks)

    # per-kernel times from the traced (non-graph) step
    prof = []
    for _ in range(max(1, args.profile_steps)):
        prof.append(sim.profile_step())
    avg = {k: statistics.mean(p[k] for p in prof) for k in prof[0]}
    bytes_rw = 2 * w.cells * esize          # one read and one write of f per pass
    fused_yz = avg["drift_y"] < 0.02 * avg["drift_z"]
    if fused_yz:                            # z and y drifts in one pass (slot 1)
        avg["drift_yz"] = avg.pop("drift_z")
        avg.pop("drift_y")
        fams = {"kick6": bytes_rw, "drift_yz": bytes_rw, "drift_x": bytes_rw}
    else:
        fams = {"kick6": bytes_rw, "drift_z": bytes_rw, "drift_y": bytes_rw, "drift_x": bytes_rw}
    dominant = max(fams, key=lambda k: avg[k])
    peak, peak_src = load_peaks()
    achieved = fams[dominant] / (avg[dominant] / 1e3) / 1e9
    kernel_names = {"kick6": "k_kick6", "drift_z": "k_drift_fast", "drift_y": "k_drift_fast",
                    "drift_yz": "k_drift_yz", "drift_x": "k_drift_fast"}
    roofline = {
        "bound": "hbm", "kernel": kernel_names[dominant], "pass": dominant,
        "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": load_traffic(dominant),
        "algorithmic_bytes_per_launch": fams[dominant],
        "kernel_ms": {k: round(v, 4) for k, v in avg.items()},
        "step_bytes_algorithmic": len(fams) * bytes_rw,
        "step_hbm_frac": round(len(fams) * bytes_rw / (avg["step"] / 1e3) / 1e9 / peak, 4),
        # the step against the bandwidth bound of the three-pass plan (24 B
        # per cell for FP32) and of the method's floor (f read and written
        # once per step, 8 B per cell)
        "step_frac_of_3pass_bound": round(3 * bytes_rw / (avg["step"] / 1e3) / 1e9 / peak, 4),
        "step_frac_of_1pass_floor": round(bytes_rw / (avg["step"] / 1e3) / 1e9 / peak, 4),
    }

    # end to end through the host-buffer entry point: every step copies its
    # input f from pinned host memory and reads back the simulated time
    e2e = None
    if args.e2e_steps > 0 and f0 is not None:
        host_in = torch.from_numpy(f0).pin_memory()
        e2e_t = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sim.step_host(host_in, 1)
            t1 = time.perf_counter()
            if i:                                   # first call: warm-up
                e2e_t.append(t1 - t0)
        e2e_ms = ranks.max(1e3 * statistics.mean(e2e_t))
        e2e = {"value": ranks.world * w.cells / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": w.cells * esize, "d2h_bytes_per_step": 64,
               "ms_per_step": round(e2e_ms, 3)}
    sim.close()
    del f

    # adjoint / forward time per step on the fixed-dt workload of the same
    # grid (the adjoint step replays its forward step, then reverses it)
    # the FP64-storage workload (16^3 x 16^3 Landau box), same timing rules
    fp64 = None
    if args.fp64_steps > 0 and w.dtype == "f32":
        fp64 = time_fp64(args, dev, stream, ranks)

    adjoint = None
    if args.adjoint_steps > 0:
        adjoint = time_adjoint(args, dev, stream)

    cpu = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline and f0 is not None:
        rate, full_s, desc = oracle_step_rate(w, f0, args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": desc}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ranks.world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if w.dtype == "f32" else "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n) + list(w.nv), "cells": w.cells,
                   "steps_timed": args.steps, "f_bytes": w.cells * esize,
                   "l2": "inputs larger than L2 (f is %.1f GB)" % (w.cells * esize / 1e9),
                   "parallelism": "replicas" if ranks.world > 1 else "single GPU"},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
        "adjoint": adjoint, "fp64": fp64, "cpu_baseline": cpu,
    }
    return out


def time_fp64(args, dev, stream, ranks):
    """Cell-updates/s of the FP64-storage Landau workload (16^3 x 16^3), timed
    like the main line (graph replay, CUDA events, warm-up excluded)."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.landau_c1()
    f = torch.from_numpy(I.initial_condition(w)).to(dev)
    sim = VlasovPoisson(config_of(w), f, stream)
    sim.step(3)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.fp64_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ranks.max(e0.elapsed_time(e1)) / args.fp64_steps
    sim.close()
    return {"workload": w.name, "dtype": "f64", "ms_per_step": round(ms, 4),
            "value": ranks.world * w.cells / (ms / 1e3), "unit": UNIT,
            "note": "f is 134 MB (near L2 size); FP64 register kernels for lines of 16"}


def time_adjoint(args, dev, stream):
    import torch
    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.WORKLOADS[args.adjoint_workload]()
    if w.cells * (4 if w.dtype == "f32" else 8) > HOST_F_LIMIT:
        f = device_initial_condition(w, dev, torch.float32 if w.dtype == "f32" else torch.float64)
    else:
        f = torch.from_numpy(I.initial_condition(w)).to(dev)
    sim = VlasovPoisson(config_of(w), f, stream)
    k = args.adjoint_steps
    sim.step(3)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(k)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fwd = e0.elapsed_time(e1) / k
    f_start = f.clone()
    g_start = sim.field()[2]
    lam_f = torch.zeros_like(f)
    lam_g = torch.zeros_like(g_start)
    sim.functional(0, lam_f)
    sim.adjoint_step(f_start, g_start, lam_f, lam_g)       # allocates its scratch
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(k):
        sim.adjoint_step(f_start, g_start, lam_f, lam_g)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    adj = e0.elapsed_time(e1) / k
    sim.close()
    return {"workload": w.name, "forward_ms_per_step": round(fwd, 3),
            "adjoint_ms_per_step": round(adj, 3), "ratio": round(adj / fwd, 3),
            "note": "adjoint step = replay of its forward step keeping the sweep inputs it cannot "
                    "recompute locally + 9 adjoint sweeps + field adjoint; the recompute of the "
                    "step-start states from the checkpoints is not included"}


def run_reference(args, ranks: Ranks):
    import numpy as np
    from paper_1206_6152_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]()
    if ranks.rank != 0:
        return None
    f0 = I.initial_condition(w)
    fraction = args.cpu_sample
    # each step a bounded sample: the density timed on the kick's planes
    # (the field solve takes the whole density, computed once here, untimed),
    # so that a long --steps run stays within minutes
    rho_full = oracle_density(w, f0)
    for _ in range(args.warmup):
        oracle_step_rate(w, f0, fraction, rho_full)
    rates, fulls = [], []
    desc = ""
    for _ in range(args.steps):
        r, full, desc = oracle_step_rate(w, f0, fraction, rho_full)
        rates.append(r)
        fulls.append(full)
    ms = 1e3 * statistics.mean(fulls)
    value = w.cells / (ms / 1e3)
    cpu = {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
           "sample": desc}
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n) + list(w.nv), "cells": w.cells},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    ranks = Ranks()
    try:
        if args.impl == "reference":
            out = run_reference(args, ranks)
        else:
            out = run_ours(args, ranks)
        if ranks.rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
    finally:
        ranks.close()


if __name__ == "__main__":
    main()
