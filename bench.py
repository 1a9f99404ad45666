#!/usr/bin/env python
"""Throughput of the 6D split step: 6D cell-updates per second.

Default workload: the 48^3 x 48^3 FP32 box (1.22e10 cells, 49 GB of f),
synthetic seeded Maxwellian with eight random-phase density modes, periodic,
adaptive dt.  A step is one whole split step of the hot path: half kick (3
velocity sweeps), drift (3 position sweeps), density, FFT Poisson solve,
force, dt, half kick (the steady-state passes fuse the two half kicks of
consecutive steps).  Besides the headline the line carries the 32^3 x 32^3
box in FP32 and in FP64 storage (the same grid, the precision comparison)
and the adjoint/forward time per step of the 32^6 and 48^6 fixed-dt boxes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica on its own GPU (the path has no exchange step); value is
the sum over ranks of the cells updated divided by the slowest rank's time.
The reference arm times the FP64 CPU oracle on the host cores on a bounded
sample of one split step of the same workload.
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


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="jeans48_modes8")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--profile-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--adjoint-steps", type=int, default=3)
    p.add_argument("--adjoint-workloads", default="jeans32_modes3,jeans48_modes8")
    p.add_argument("--fp64-steps", type=int, default=20)
    p.add_argument("--extra-workload", default="jeans32_f32",
                   help="second FP32 line, also timed in FP64 storage ('' for none)")
    p.add_argument("--cpu-sample", type=float, default=1.0 / 64)
    p.add_argument("--slabs", type=int, default=2,
                   help="x slabs of the slab-decomposition leg (all in this process)")
    p.add_argument("--slab-workload", default="jeans32_f32")
    p.add_argument("--slab-steps", type=int, default=5, help="0: no slab-decomposition leg")
    p.add_argument("--record-traffic", metavar="CSV", default="",
                   help="write profiles/traffic.json entries for --workload from an ncu --csv "
                        "launch list with dram__bytes_read.sum and dram__bytes_write.sum, taken "
                        "on the current kernel sources; no GPU work")
    return p.parse_args(argv)


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


class HostSource:
    """FP64 pieces of a workload's initial condition for the oracle's samples:
    slices of a host array f0 when there is one, otherwise products of the
    two FP64 factors rho(x) M(v) of a separable initial condition (the values
    initial_condition() rounds once), so that a 49 GB f needs no host copy."""

    def __init__(self, w, f0=None):
        self.w = w
        self.f0 = f0
        if f0 is None:
            from paper_1206_6152_gb300 import inputs as I
            if w.ic in ("king", "king2"):
                raise ValueError("a King initial condition is not separable: pass f0")
            self.rho_x, self.mv = I.factors(w)

    def planes(self, lo: int, hi: int):
        """f[lo:hi] (x planes), FP64."""
        import numpy as np
        w = self.w
        if self.f0 is not None:
            return np.ascontiguousarray(self.f0[lo:hi], dtype=np.float64)
        nyz = w.n[1] * w.n[2]
        return np.multiply.outer(self.rho_x[lo * nyz:hi * nyz], self.mv).reshape(
            (hi - lo,) + tuple(w.n[1:]) + tuple(w.nv))

    def vcols(self, svx: int):
        """f[:, :, :, :svx] (the first svx vx columns of every velocity cube), FP64."""
        import numpy as np
        w = self.w
        if self.f0 is not None:
            return np.ascontiguousarray(self.f0[:, :, :, :svx], dtype=np.float64)
        m = self.mv.reshape(w.nv)[:svx].reshape(-1)
        return np.multiply.outer(self.rho_x, m).reshape(tuple(w.n) + (svx,) + tuple(w.nv[1:]))

    def density(self):
        """rho of the whole grid: the oracle's density slab by slab (host
        array), or rho_x sum(M) dV_v from the factors."""
        import numpy as np
        from oracle import vp_oracle as O
        w = self.w
        if self.f0 is None:
            return (self.rho_x * (self.mv.sum() * O.Grid.of(w).dvol_v)).reshape(w.n)
        grid = O.Grid.of(w)
        slab = O.Grid((1,) + tuple(w.n[1:]), grid.nv, grid.lo, grid.hi, grid.vlo, grid.vhi)
        return np.concatenate([O.density(self.planes(i, i + 1), slab) for i in range(w.n[0])])


def oracle_density(w, f0_np):
    """The oracle's density of the whole grid, slab by slab."""
    return HostSource(w, f0_np).density()


def oracle_step_rate(w, src, fraction: float, rho_full=None):
    """Times the FP64 oracle on a sample of one split step of workload w and
    scales it to the whole step: the density of a fraction of the x planes
    (scaled), the Poisson solve and force on the whole density rho_full
    (computed here, untimed, when not given), the six velocity sweeps on the
    cubes of the same x planes and the three position sweeps on the whole
    lines of a fraction of the velocity cells.  src: a HostSource, or a host
    array of f.  Returns (cell-updates/s of the whole step, seconds per whole
    step, description, seconds the sample took)."""
    import numpy as np
    from oracle import vp_oracle as O
    if not isinstance(src, HostSource):
        src = HostSource(w, src)
    grid = O.Grid.of(w)
    nx, ny, nz = w.n
    nvx, nvy, nvz = w.nv
    sx = max(1, min(nx, int(round(fraction * nx))))
    if rho_full is None:
        rho_full = src.density()
    wall0 = time.perf_counter()
    fk = src.planes(0, sx)
    qk = fk.size / w.cells
    slab = O.Grid((sx, ny, nz), grid.nv, grid.lo, grid.hi, grid.vlo, grid.vhi)
    t0 = time.perf_counter()
    O.density(fk, slab)
    t_dens = (time.perf_counter() - t0) / qk
    t0 = time.perf_counter()
    phi = O.poisson(rho_full, grid, w.G, w.poisson_bc)
    g = O.force(phi, grid, w.poisson_bc)
    dt = O.timestep(g, grid, w.courant) if w.dt_fixed <= 0 else w.dt_fixed
    t_field = time.perf_counter() - t0
    # velocity sweeps on a block of whole cubes (both half kicks)
    t0 = time.perf_counter()
    for _ in range(2):
        for a in range(3):
            O.sweep(fk, 3 + a, np.ascontiguousarray(g[a][:sx]), dt / 2, grid.dv[a], False)
    t_kick = time.perf_counter() - t0
    del fk
    # position sweeps on the whole lines of a block of velocity cells
    svx = max(1, min(nvx, int(round(fraction * nvx))))
    fd = src.vcols(svx)
    qd = fd.size / w.cells
    t0 = time.perf_counter()
    for a in (2, 1, 0):
        O.sweep(fd, a, grid.vc(a)[:svx] if a == 0 else grid.vc(a), dt, grid.dx[a],
                w.space_bc == "periodic")
    t_drift = time.perf_counter() - t0
    del fd
    measured = time.perf_counter() - wall0
    full = t_dens + t_field + t_kick / qk + t_drift / qd
    desc = (f"FP64 oracle, one split step of {w.name}: density timed on {sx} of {nx} x planes "
            f"and scaled, the Poisson solve timed in full; the 6 velocity sweeps timed on "
            f"{sx * ny * nz} of {nx * ny * nz} velocity cubes ({qk:.4f}) and the 3 position sweeps "
            f"on the lines of {svx * nvy * nvz} of {nvx * nvy * nvz} velocity cells ({qd:.4f}), each "
            f"scaled by its fraction; the sample took {measured:.1f} s, the whole step "
            f"{full:.1f} s")
    return w.cells / full, full, desc, measured


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

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


def make_f(w, dev, dtype=None):
    """(f on the device, the host array it came from or None): separable
    initial conditions are built on the device from their two factors, the
    King spheres on the host."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    tdt = dtype or (torch.float32 if w.dtype == "f32" else torch.float64)
    if w.ic not in ("king", "king2"):
        return device_initial_condition(w, dev, tdt), None
    f0 = I.initial_condition(w, np_dtype(tdt))
    return torch.from_numpy(f0).to(dev), f0


def np_dtype(tdt):
    import numpy as np
    import torch
    return np.float32 if tdt == torch.float32 else np.float64


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("vp_sweep.cu", "vp_sweep_fast.cu", "vp_kick_big.cu", "vp_fast_line.cuh",
                  "vp_line.cuh", "vp_device.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1206_6152_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        ent = d[key]
        if ent.get("source_hash") != kernel_source_hash():
            return None
        return float(ent["dram_bytes_per_launch_full"])
    except Exception:
        return None


# the forward passes of one steady-state step: (profile slot, kernel, traffic key)
PASSES_BIG = (("kick_a", "k_kick_pass_a", "{w}:kick_a"), ("kick_b", "k_kick_pass_b", "{w}:kick_b"),
              ("kick_c", "k_kick_pass_c", "{w}:kick_c"), ("drift_z", "k_drift_fast", "{w}:drift_z"),
              ("drift_y", "k_drift_fast", "{w}:drift_y"), ("drift_x", "k_drift_fast", "{w}:drift_x"))
PASSES_FUSED = (("kick6", "k_kick6", "{w}:kick6"), ("drift_yz", "k_drift_yz", "{w}:drift_yz"),
                ("drift_x", "k_drift_fast", "{w}:drift_x"))


def _ncu_launches(csv_path):
    """[(kernel name, {metric: value in bytes or ns})] in launch order from an
    ncu --csv log."""
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0,
             "usecond": 1e3, "msecond": 1e6, "second": 1e9}
    launches, hdr = {}, None
    with open(csv_path) as fh:
        for row in csv.reader(fh):
            if row and row[0] == "ID":
                hdr = row
                continue
            if not hdr or len(row) != len(hdr):
                continue
            d = dict(zip(hdr, row))
            ent = launches.setdefault(int(d["ID"]), (d["Kernel Name"], {}))
            ent[1][d["Metric Name"]] = float(d["Metric Value"].replace(",", "")) * scale.get(
                d["Metric Unit"], 1.0)
    return [launches[i] for i in sorted(launches)]


def record_traffic(csv_path, workload):
    """profiles/traffic.json entries of workload's forward passes: DRAM bytes
    read + written per launch, averaged over the captured launches of each
    pass (the z and y drifts of the same kernel told apart by their order)."""
    launches = _ncu_launches(csv_path)
    slots = {}
    zy = 0
    for name, m in launches:
        if "dram__bytes_read.sum" not in m:
            continue
        if "k_kick_pass_a" in name: slot = "kick_a"
        elif "k_kick_pass_b" in name: slot = "kick_b"
        elif "k_kick_pass_c" in name: slot = "kick_c"
        elif "k_kick6" in name: slot = "kick6"
        elif "k_drift_yz" in name: slot = "drift_yz"
        elif "k_drift_fast" in name and name.replace(" ", "").split(",")[3].startswith("1>"):
            slot = "drift_x"
        elif "k_drift_fast" in name:
            slot = ("drift_z", "drift_y")[zy % 2]
            zy += 1
        else:
            continue
        slots.setdefault(slot, []).append(m)
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            out = json.load(fh)
    except Exception:
        out = {}
    h = kernel_source_hash()
    for slot, ms in slots.items():
        rw = [m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"] for m in ms]
        out[f"{workload}:{slot}"] = {
            "source_hash": h, "launches": len(ms),
            "dram_bytes_read": statistics.mean(m["dram__bytes_read.sum"] for m in ms),
            "dram_bytes_write": statistics.mean(m["dram__bytes_write.sum"] for m in ms),
            "dram_bytes_per_launch_full": statistics.mean(rw),
            "duration_us_under_ncu": statistics.mean(m.get("gpu__time_duration.sum", 0.0) for m in ms) / 1e3,
            "captured_on": f"{workload} at full size, ncu launch list ({os.path.basename(csv_path)})"}
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    return out


def roofline_of(w, avg, esize):
    """The step's forward passes from one profiled step (CUDA events on the
    context's stream): algorithmic bytes per launch (f read once and written
    once, 2 x cells x element size), achieved GB/s, and the dominant (longest)
    kernel against the measured HBM peak."""
    bytes_rw = 2 * w.cells * esize
    avg = dict(avg)
    # the kick: three slab passes (48^3 cubes) or one cube pass
    kicks = PASSES_BIG[:3] if avg.get("kick_a", 0.0) > 0.0 else PASSES_FUSED[:1]
    if avg["drift_y"] < 0.02 * avg["drift_z"]:          # z and y drifts fused (slot 1)
        avg["drift_yz"] = avg["drift_z"]
        drifts = PASSES_FUSED[1:]
    else:
        drifts = PASSES_BIG[3:]
    passes = kicks + drifts
    peak, peak_src = load_peaks()
    per = {slot: {"kernel": k, "ms": round(avg[slot], 4),
                  "achieved_gbs": round(bytes_rw / (avg[slot] / 1e3) / 1e9, 1)} for slot, k, _ in passes}
    slot, kern, tkey = max(passes, key=lambda p: avg[p[0]])
    achieved = bytes_rw / (avg[slot] / 1e3) / 1e9
    npass = len(passes)
    return {
        "bound": "hbm", "kernel": kern, "pass": slot,
        "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": load_traffic(tkey.format(w=w.name)),
        "algorithmic_bytes_per_launch": bytes_rw,
        "passes": per,
        "kernel_ms": {k: round(v, 4) for k, v in avg.items()},
        "step_bytes_algorithmic": npass * bytes_rw,
        "step_hbm_frac": round(npass * bytes_rw / (avg["step"] / 1e3) / 1e9 / peak, 4),
        # the step against the method's floor (f read and written once per
        # step, 8 B per cell for FP32)
        "step_frac_of_1pass_floor": round(bytes_rw / (avg["step"] / 1e3) / 1e9 / peak, 4),
    }


def timed_steps(sim, steps, warmup, dev, stream, ranks, clocks=None):
    """Graph-replayed split steps between two CUDA events on the context's
    stream, after the warm-up; returns (ms, kernel launches)."""
    import torch
    sim.step(max(warmup, 3))
    torch.cuda.synchronize(dev)
    k0 = sim.kernels_launched()
    ranks.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ranks.barrier()
    return e0.elapsed_time(e1), sim.kernels_launched() - k0


def profile(sim, n):
    prof = [sim.profile_step() for _ in range(max(1, n))]
    return {k: statistics.mean(p[k] for p in prof) for k in prof[0]}


def run_ours(args, ranks: Ranks):
    import torch

    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of

    w = I.WORKLOADS[args.workload]()
    dev = torch.device("cuda", ranks.local)
    torch.cuda.set_device(dev)
    f, f0 = make_f(w, dev)
    stream = torch.cuda.current_stream(dev)
    sim = VlasovPoisson(config_of(w), f, stream)
    esize = f.element_size()

    clocks = Clocks(dev.index if dev.index is not None else 0)
    ms, launches = timed_steps(sim, args.steps, args.warmup, dev, stream, ranks, clocks)
    clk = clocks.stop()
    ms_max, value = aggregate(ms, w.cells, args.steps, ranks)
    roofline = roofline_of(w, profile(sim, args.profile_steps), esize)

    # end to end through the host-buffer entry point: every step copies its
    # input f from pinned host memory, runs the step and reads the stepped f
    # back into the same buffer
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
        host.copy_(f)
        e2e_t = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sim.step_host(host, 1, host)
            t1 = time.perf_counter()
            if i:                                   # first call: warm-up
                e2e_t.append(t1 - t0)
        del host
        release = getattr(torch._C, "_host_emptyCache", None)    # torch's pinned-memory cache
        if release is not None:
            release()
        e2e_ms = ranks.max(1e3 * statistics.mean(e2e_t))
        e2e = {"value": ranks.world * w.cells / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": w.cells * esize, "d2h_bytes_per_step": w.cells * esize,
               "ms_per_step": round(e2e_ms, 3),
               "note": "vp_step_host: f from pinned host memory, one split step, f back to the "
                       "same buffer"}
    sim.close()
    del f
    torch.cuda.empty_cache()        # the library allocates outside torch's cache

    extra = None
    if args.extra_workload not in ("", "none") and args.extra_workload != args.workload:
        extra = time_extra(args, dev, stream, ranks)

    slabs = None
    if args.slab_steps > 0 and args.slabs > 0 and ranks.world == 1:
        slabs = time_slabs(args, dev, stream)

    adjoint = []
    if args.adjoint_steps > 0:
        for aw in [x for x in args.adjoint_workloads.split(",") if x]:
            adjoint.append(time_adjoint(args, aw, dev, stream))

    cpu = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline:
        rate, full_s, desc, _ = oracle_step_rate(w, HostSource(w, f0), args.cpu_sample)
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
        "extra": extra, "slabs": slabs, "adjoint": adjoint, "cpu_baseline": cpu,
    }
    return out


def time_extra(args, dev, stream, ranks):
    """A second workload timed like the headline in FP32 and in FP64 storage
    (the same grid): the precision comparison of the metric."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.WORKLOADS[args.extra_workload]()
    out = {"workload": w.name, "grid": list(w.n) + list(w.nv), "cells": w.cells}
    for tdt, key, steps in ((torch.float32, "f32", args.steps), (torch.float64, "f64", args.fp64_steps)):
        if steps <= 0:
            continue
        f, _ = make_f(w, dev, tdt)
        sim = VlasovPoisson(config_of(w, tdt), f, stream)
        ms, launches = timed_steps(sim, steps, 3, dev, stream, ranks)
        ms_max, value = aggregate(ms, w.cells, steps, ranks)
        line = {"value": value, "unit": UNIT, "ms_per_step": round(ms_max / steps, 4),
                "steps": steps, "f_bytes": w.cells * f.element_size(), "gpu_launches": launches}
        if key == "f32":
            line["roofline"] = roofline_of(w, profile(sim, args.profile_steps), f.element_size())
        out[key] = line
        sim.close()
        del f
        torch.cuda.empty_cache()
    return out


def time_slabs(args, dev, stream):
    """The split step over x slabs of position space (sharded.py) with all
    slabs in this process on one GPU, exchanging by direct copies: the
    single-context step plus what the decomposition adds (the ghosted x
    drift, the halo planes, the reduction of the line maxima, the gathered
    density and a field solve per slab, host-side orchestration and one host
    read of dt per step).  Wall clock between synchronisations; the ghosted
    x drift alone between CUDA events on the slabs' stream."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.sharded import LibrarySlab, LocalExchange, ShardedStep
    from paper_1206_6152_gb300.vlasov import config_of
    w = I.WORKLOADS[args.slab_workload]()
    R = args.slabs
    if w.n[0] % R:
        return {"workload": w.name, "unavailable": f"{w.n[0]} x planes do not split into {R} slabs"}
    torch.cuda.empty_cache()
    f, _ = make_f(w, dev)
    cfg = config_of(w)
    nx = w.n[0] // R
    slabs = [LibrarySlab(cfg, r * nx, f[r * nx:(r + 1) * nx], stream) for r in range(R)]
    try:
        step = ShardedStep(slabs, LocalExchange())
        k = args.slab_steps
        step.step(3)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step.step(k)
        torch.cuda.synchronize(dev)
        ms = 1e3 * (time.perf_counter() - t0) / k
        # the ghosted x drift of one slab, timed alone
        s0 = slabs[0]
        G = step.nghost(step.dt)
        lo, hi = s0.planes(nx - G, nx), s0.planes(0, G)
        lmax = s0.line_max_x()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.drift_x(step.dt, lo, hi, G, lmax)
        e0.record(stream)
        for _ in range(k):
            s0.drift_x(step.dt, lo, hi, G, lmax)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        dx_ms = e0.elapsed_time(e1) / k
        slab_bytes = 2 * (w.cells // R) * f.element_size()
        peak, _ = load_peaks()
        return {"workload": w.name, "slabs": R, "planes_per_slab": nx, "ghost_planes": G,
                "ms_per_step": round(ms, 3), "value": w.cells / (ms / 1e3), "unit": UNIT,
                "drift_x_ghosted": {"ms": round(dx_ms, 4),
                                    "achieved_gbs": round(slab_bytes / (dx_ms / 1e3) / 1e9, 1),
                                    "frac": round(slab_bytes / (dx_ms / 1e3) / 1e9 / peak, 4),
                                    "bytes": "f of the slab read and written once (ghost reads "
                                             "not counted)"},
                "note": "all slabs on one GPU in one process (direct copies for the exchanges); "
                        "wall clock per step between synchronisations"}
    finally:
        for s in slabs:
            s.close()
        del f
        torch.cuda.empty_cache()


def time_adjoint(args, name, dev, stream):
    """Adjoint / forward time per step of a fixed-dt workload (the adjoint
    step replays its forward step, then reverses it)."""
    import torch
    from paper_1206_6152_gb300 import inputs as I
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.WORKLOADS[name]()
    torch.cuda.empty_cache()
    f, _ = make_f(w, dev)
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
    # the step-start state is the context's own f, which the adjoint step
    # leaves unchanged, as in the checkpointed trajectory (adjoint.py): the
    # memory a copy would take goes to the adjoint's scratch states
    f_start = f
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
    del f, f_start, lam_f
    torch.cuda.empty_cache()
    return {"workload": w.name, "forward_ms_per_step": round(fwd, 3),
            "adjoint_ms_per_step": round(adj, 3), "ratio": round(adj / fwd, 3),
            "note": "adjoint step = replay of its forward step keeping the sweep inputs it cannot "
                    "recompute locally + 9 adjoint sweeps + field adjoint; the step-start state is "
                    "the context's own f; the recompute of the step-start states from the "
                    "checkpoints is not included"}


def run_reference(args, ranks: Ranks):
    """The FP64 oracle on the host cores; each step is the bounded sample of
    one split step (oracle_step_rate): ms_per_step is the time the sample
    took, value the cell-updates/s of the whole step it stands for."""
    from paper_1206_6152_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]()
    if ranks.rank != 0:
        return None
    f0 = None
    if w.ic in ("king", "king2"):
        f0 = I.initial_condition(w)
    src = HostSource(w, f0)
    rho_full = src.density()
    for _ in range(args.warmup):
        oracle_step_rate(w, src, args.cpu_sample, rho_full)
    fulls, measured = [], []
    desc = ""
    for _ in range(args.steps):
        _, full, desc, meas = oracle_step_rate(w, src, args.cpu_sample, rho_full)
        fulls.append(full)
        measured.append(meas)
    value = w.cells / statistics.mean(fulls)
    cpu = {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
           "sample": desc}
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(measured),
        "ms_per_step_whole_step_estimate": 1e3 * statistics.mean(fulls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n) + list(w.nv), "cells": w.cells},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.record_traffic:
        record_traffic(args.record_traffic, args.workload)
        return
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
