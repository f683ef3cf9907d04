#!/usr/bin/env python
"""Benchmark of the GB300 explicit EM-PIC hot path (KEMPIC-3D cycle: Faraday half
step, fused gather + Boris + zigzag deposit, Faraday half step, Ampere).

Headline workload: thermal plasma, 256^3 periodic cells, dx = 0.2 c/w_p, 32 electrons
per cell (536,870,912 particles) at uniform random positions with Maxwellian momenta
u_th = 0.1 c (drawn on the device: torch's Philox generator, seed 1238), immobile ions,
dt = 0.5 x Courant, FP32 bulk; the FP64 GPU path runs the same inputs.  One step = one
full PIC cycle over every particle and cell.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbpic|reference]

Under torchrun every rank runs its own replica (the method has no exchange step on one
GPU; replicas only) and the value is the sum over ranks of particle-steps divided by
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import multiprocessing
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle pushes/s incl. deposit (FP32 vs FP64 GPU), % HBM roofline"
UNIT = "particle-steps/s"
# the headline: the largest single-GPU workload (256^3 x 32 per cell, u_th = 0.1); the
# 128^3 x 64 thermal plasma (u_th = 0.05) is timed as an extra and selectable here
WORKLOADS = {
    "stress256": dict(name="stress256", n=(256, 256, 256), d=0.2, ppc=32, u_th=0.1, seed=1238),
    "thermal128": dict(name="thermal128", n=(128, 128, 128), d=0.2, ppc=64, u_th=0.05, seed=1235),
}
# algorithmic bytes (what the method must move; sorting, ghosts and the fixed-point
# width of J are overheads counted against the achieved fraction)
PART_BYTES = {"f32": 60, "f64": 112}       # read cell + 3 offsets + 3 momenta + w, write all but w
TILE_GRID_BYTES = {"f32": 36, "f64": 72}   # gather reads E, B (24 B) + deposit writes J (12 B) per cell
STEP_GRID_BYTES = {"f32": 108, "f64": 216}  # + Yee: read E, B, J, write E, B, zero J (72 B)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gbpic", choices=["gbpic", "reference"])
    p.add_argument("--workload", default="stress256", choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the other workloads and the adjoint cost")
    p.add_argument("--adjoint-only", type=int, default=0,
                   help="only time the FP64 checkpointed adjoint of the differentiable run over this many steps")
    p.add_argument("--adjoint-prec", default="f64", choices=["f32", "f64", "both"],
                   help="precision of the --adjoint-only timing")
    p.add_argument("--waveguide", type=int, default=0,
                   help="run the first N grids of the TE10 waveguide convergence study (FP64) and exit")
    p.add_argument("--waveguide-fp32", action="store_true", help="the waveguide study on the FP32 path")
    p.add_argument("--small", action="store_true", help="32^3 cells instead of the headline grid (smoke)")
    p.add_argument("--cells", type=int, default=0, help="cells per dimension of the headline workload (profiling)")
    p.add_argument("--ppc", type=int, default=0, help="electrons per cell of the headline workload (profiling)")
    p.add_argument("--deposit", default="zigzag", choices=["zigzag", "esirkepov"],
                   help="current deposit of the headline run (profiling the variants)")
    p.add_argument("--shape", default="cic", choices=["cic", "tsc"], help="particle shape of the headline run")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


_C_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)


def kernel_source_hash(root=None):
    """Hash of the tile kernel's source with comments dropped and whitespace collapsed:
    a committed ncu capture stays valid across comment and layout edits."""
    h = hashlib.sha256()
    for name in ("push.cu", "push_common.cuh", "pic_internal.cuh"):
        with open(os.path.join(root or ROOT, "paper_2609_16575_gb300", "csrc", name)) as f:
            text = f.read()
        code = _C_TOKENS.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload, n_particles):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    try:
        with open(path) as f:
            prof = json.load(f)
    except Exception:
        return None
    if prof.get("source_sha") != kernel_source_hash():
        return None
    per_particle = prof.get("dram_bytes_per_particle")
    return None if per_particle is None else per_particle * n_particles


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            self.tmp.flush()
            rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def workload_spec(args):
    """The headline workload, with the profiling overrides of the grid and ppc."""
    spec = dict(WORKLOADS[args.workload])
    if args.small:
        spec["n"] = (32, 32, 32)
    elif args.cells:
        spec["n"] = (args.cells,) * 3
    if args.ppc:
        spec["ppc"] = args.ppc
    return spec


def describe(spec):
    n = spec["n"]
    npart = n[0] * n[1] * n[2] * spec["ppc"]
    return (f"thermal plasma {n[0]}x{n[1]}x{n[2]} periodic cells, dx={spec['d']}, {spec['ppc']} electrons per cell "
            f"({npart:,}), u_th={spec['u_th']}, immobile ions, dt=0.5 Courant; inputs drawn on the device "
            f"(Philox, seed {spec['seed']} + rank)")


def _oracle_sample(q, barrier, n, d, ppc, u_th, seed, warmup, steps):
    """One host process: the FP64 oracle, as it stands, on an n^3 thermal sample."""
    import oracle
    from paper_2609_16575_gb300 import workloads as W

    wl = W.thermal((n, n, n), d, ppc, u_th, seed=seed)
    sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
    F = oracle.empty_fields(wl.n)
    oracle.run(wl.n, wl.d, wl.dt, F, sp, max(int(warmup), 1))    # page-in, library load
    barrier.wait()
    t0 = time.monotonic()
    oracle.run(wl.n, wl.d, wl.dt, F, sp, steps)
    t1 = time.monotonic()
    q.put((wl.nparticles, steps, t0, t1))


def oracle_rate(workers, spec, n=32, warmup=1, steps=10):
    """Particle-steps/s of `workers` concurrent single-thread oracle processes (spawned,
    each on its own seeded n^3 sample of the workload's ppc and u_th, all started
    together behind a barrier): total particle-steps over the wall time from the first
    start to the last end."""
    import oracle

    oracle.build()
    mp = multiprocessing.get_context("spawn")
    q, bar = mp.Queue(), mp.Barrier(workers)
    procs = [mp.Process(target=_oracle_sample,
                        args=(q, bar, n, spec["d"], spec["ppc"], spec["u_th"], spec["seed"] + i, warmup, steps))
             for i in range(workers)]
    for p in procs:
        p.start()
    res = [q.get(timeout=1800) for _ in procs]
    for p in procs:
        p.join()
    wall = max(r[3] for r in res) - min(r[2] for r in res)
    total = sum(r[0] * r[1] for r in res)
    return total / wall, wall, res[0][0]


def host_memory_available():
    """Bytes of host memory available to this process: MemAvailable, capped by a cgroup
    limit when there is one."""
    avail = float("inf")
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            v = open(path).read().strip()
            if v.isdigit():
                avail = min(avail, int(v))
        except OSError:
            pass
    return avail


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(spec, steps=10, n=32):
    """The FP64 oracle, as it stands, on a bounded sample of the workload (a 32^3 box at
    the workload's ppc and u_th, `steps` cycles): on one host core and on every core of
    the host (one process per core, each on its own sample)."""
    v1, w1, npart = oracle_rate(1, spec, n, 1, steps)
    cores = host_cores()
    vn, wn, _ = oracle_rate(cores, spec, n, 1, steps) if cores > 1 else (v1, w1, npart)
    sample = (f"thermal {n}^3 cells x {spec['ppc']} ppc, u_th={spec['u_th']} ({npart:,} particles per process), "
              f"{steps} cycles, FP64 oracle")
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample + f", {cores} processes (one per host core, nproc = {cores})",
            "seconds": round(wn, 2),
            "single_core": {"value": v1, "unit": UNIT, "cores": 1, "seconds": round(w1, 2)}}


def time_steps(ctx, torch, steps, kernels=True):
    """CUDA-event time (ms) of `steps` cycles on the context's stream, with the library's
    per-kernel times (kernels=True; per-launch events, and the cycles run launch by
    launch) or without them (the library may then replay the cycles as a CUDA graph)."""
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if kernels:
        ctx.set_timing(True)
        ctx.kernel_times()
    a.record(st)
    ctx.step(steps)
    b.record(st)
    torch.cuda.synchronize()
    kt = {}
    if kernels:
        kt = ctx.kernel_times()
        ctx.set_timing(False)
    return a.elapsed_time(b), kt


def kernel_table(kt):
    return {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items() if v[0]}


def thermal_context(torch, gbpic, W, spec, prec):
    """A context holding the thermal workload `spec`, inputs drawn on the device."""
    X, U, w, dt = W.thermal_device(torch, spec["n"], spec["d"], spec["ppc"], spec["u_th"], spec["seed"])
    ctx = gbpic.Context(spec["n"], (spec["d"],) * 3, dt, precision=prec, rho_ion=1.0,
                        device=torch.cuda.current_device())
    ctx.load_species(-1.0, 1.0, X, U, w, True)
    npart = int(w.shape[0])
    del X, U, w
    return ctx, npart


def other_workloads(torch, peak, peak_kind):
    """Throughput on the other workload shapes: the 128^3 x 64 thermal plasma (FP32, its
    own roofline), the cold-plasma oscillation (16^3, 8 per cell, FP64 and FP32), the
    laser wakefield (512 x 128 x 128, open x, 8 per cell, FP32) timed while the pulse
    crosses the density ramp, and the thermal plasma with the current filter, with
    Esirkepov's deposit and the wakefield with a moving window."""
    from paper_2609_16575_gb300 import gbpic
    from paper_2609_16575_gb300 import workloads as W

    out = {}
    spec = WORKLOADS["thermal128"]
    ncell = spec["n"][0] ** 3
    ctx, npart = thermal_context(torch, gbpic, W, spec, gbpic.PIC_FP32)
    time_steps(ctx, torch, 5)
    steps = 20
    ms, kt = time_steps(ctx, torch, steps)
    ctx.close()
    out["thermal128_f32"] = {
        "value": npart * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "workload": describe(spec), "particles": npart,
        "roofline": roofline(kt, "f32", npart, ncell, peak, peak_kind,
                             committed_traffic("tile_push", "thermal128", npart)),
        "yee": yee_line(kt, ncell, peak), "kernels": kernel_table(kt)}

    wl = W.cold_plasma(n=16)
    for prec, name in ((gbpic.PIC_FP64, "f64"), (gbpic.PIC_FP32, "f32")):
        ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion)
        s = wl.species[0]
        ctx.load_species_array(s.q, s.m, s.P, True)
        time_steps(ctx, torch, 10, kernels=False)
        ms, _ = time_steps(ctx, torch, 200, kernels=False)
        out[f"cold_plasma_16_{name}"] = {"value": s.n * 200 / (ms / 1e3), "unit": UNIT, "steps": 200,
                                          "ms_per_step": ms / 200, "particles": s.n,
                                          "note": "launch-bound: 32,768 particles fill 8 tiles; the cycles run as "
                                                  "a replayed two-cycle CUDA graph"}
        ctx.close()

    # the laser wakefield: 1000 cycles first (the pulse peak, injected at t = 2 FWHM, has
    # then entered the density ramp), then 20 timed cycles
    wl = W.lwfa()
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion, bc_x=1)
    ctx.set_laser(*wl.laser.as_tuple())
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    del wl.species[0].P
    ctx.step(1000)
    ctx.sync()
    n0 = ctx.diagnostics()["n_alive"]
    steps = 20
    ms, kt = time_steps(ctx, torch, steps)
    d1 = ctx.diagnostics()
    ncell = wl.n[0] * wl.n[1] * wl.n[2]
    npart = 0.5 * (n0 + d1["n_alive"])
    out["lwfa_512x128x128_f32"] = {
        "value": npart * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "particles": [n0, d1["n_alive"]], "U_E": d1["U_E"], "K_half": d1["K_half"],
        "roofline": roofline(kt, "f32", npart, ncell, peak, peak_kind, None),
        "yee": yee_line(kt, ncell, peak), "kernels": kernel_table(kt),
        "note": "cycles 1001-1020: the pulse (peak at t = 2 FWHM on the source plane) is crossing the density ramp"}
    ctx.close()

    # the thermal plasma with the compensated binomial current filter (1 pass per
    # dimension and the compensator) and with Esirkepov's deposit
    for key, setup in (("thermal128_filtered_f32", lambda c: c.set_current_filter(1, True)),
                       ("thermal128_esirkepov_f32", lambda c: c.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV)),
                       ("thermal128_tsc_f32", lambda c: c.set_shape(gbpic.PIC_SHAPE_TSC))):
        X, U, w, dt = W.thermal_device(torch, spec["n"], spec["d"], spec["ppc"], spec["u_th"], spec["seed"])
        ctx = gbpic.Context(spec["n"], (spec["d"],) * 3, dt, precision=gbpic.PIC_FP32, rho_ion=1.0)
        setup(ctx)
        ctx.load_species(-1.0, 1.0, X, U, w, True)
        npart = int(w.shape[0])
        del X, U, w
        time_steps(ctx, torch, 3)
        steps = 10
        ms, kt = time_steps(ctx, torch, steps)
        ctx.close()
        out[key] = {"value": npart * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
                    "particles": npart, "kernels": kernel_table(kt)}
    out["thermal128_tsc_f32"]["note"] = ("quadratic (TSC) shape: 27-point gather per component and Esirkepov's "
                                         "deposit on the 4 x 4 x 4 support, every particle")
    out["thermal128_filtered_f32"]["note"] = ("'other' holds the filter: 1 binomial pass per dimension and the "
                                              "compensator, each over J")
    base = out["thermal128_f32"]["kernels"]["tile_push"]
    ek = out["thermal128_esirkepov_f32"]["kernels"]
    esk = ek.get("tile_push")
    if esk:
        # the crossers' deposit runs in its own kernel after the tile kernel
        cross = ek.get("esk_crossers", {"ms": 0.0})
        out["thermal128_esirkepov_f32"]["particle_kernels_over_zigzag"] = ((esk["ms"] + cross["ms"]) / esk["launches"]) / (
            base["ms"] / base["launches"])
        out["thermal128_esirkepov_f32"]["step_over_zigzag"] = (out["thermal128_esirkepov_f32"]["ms_per_step"] /
                                                               out["thermal128_f32"]["ms_per_step"])

    # the wakefield with the moving window: a one-cell move every ceil(dx / dt) = 3
    # cycles from the first cycle on, the new column's plasma injected at each move
    wl = W.lwfa(window_start=0)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion, bc_x=1)
    ctx.set_laser(*wl.laser.as_tuple())
    ctx.set_moving_window(*wl.window.as_tuple())
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    time_steps(ctx, torch, 3)
    n_before, m_before = ctx.diagnostics()["n_alive"], ctx.window_moves()
    steps = 30
    ms, kt = time_steps(ctx, torch, steps)
    n_after, m_after = ctx.diagnostics()["n_alive"], ctx.window_moves()
    npart = 0.5 * (n_before + n_after)
    out["lwfa_512x128x128_window_f32"] = {
        "value": npart * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "particles": [n_before, n_after], "moves": m_after - m_before, "every": wl.window.every,
        "kernels": kernel_table(kt),
        "note": "cycles 4-33 with a moving window; 'other' holds the field shift, the injection, the "
                "laser sheet and the Mur faces"}
    ctx.close()
    return out


# The TE10 waveguide of the Yee verification (section 3.2): a = 3 cm, b = a / 2, length
# 1 m, excitation 9 GHz with the envelope 1 - exp(-t / 2 periods), Courant number 0.5.
# Grids: the node counts (across a, across b, along the guide) and step counts of the
# paper's convergence table, with its errors of the steady-state E amplitude for context.
WAVEGUIDE_GRIDS = [(12, 6, 376, 1251, 4.54e-2), (23, 12, 751, 2501, 4.37e-3), (46, 23, 1501, 5001, 2.95e-3),
                   (91, 46, 3001, 10001, 3.74e-4), (181, 91, 6001, 20001, 8.41e-5)]


def _fit_wave(x, f, beta0):
    """Amplitude and wave number of f(x) = A sin(beta x - phi) (least squares over beta)."""
    import numpy as np

    def resid(beta):
        A = np.stack([np.sin(beta * x), np.cos(beta * x)], 1)
        c, *_ = np.linalg.lstsq(A, f, rcond=None)
        r = f - A @ c
        return float(r @ r), float(np.hypot(*c))

    betas = np.linspace(0.97 * beta0, 1.03 * beta0, 601)
    best = min(betas, key=lambda b: resid(b)[0])
    lo, hi = best - (betas[1] - betas[0]), best + (betas[1] - betas[0])
    for _ in range(80):   # golden-section refinement
        m1, m2 = lo + 0.382 * (hi - lo), lo + 0.618 * (hi - lo)
        if resid(m1)[0] < resid(m2)[0]:
            hi = m2
        else:
            lo = m1
    beta = 0.5 * (lo + hi)
    return resid(beta)[1], beta


def waveguide_convergence(torch, count, fp64=True):
    """The TE10 convergence study on the GPU (FP64 by default: an accuracy study that
    FP32 rounding must not limit), in units of the excitation: time in
    periods, length in free-space wavelengths (c = 1, omega = 2 pi).  The guide's length
    runs along the open x, its width a along y and its height b along z, closed by the
    wall planes y = 0 and z = 0; the port drives Ez = sin(pi y / a) on x = 0.  At the end
    of each run the steady part of Ez along the guide's axis (from L/16 to where the
    envelope has risen, 1 - exp(-10)) is fitted with A sin(beta x - phi): A against the
    port amplitude at the probe's y, beta against the continuous guide's
    sqrt(omega^2 - (pi / a)^2); rates are least-squares slopes against the cell diagonal."""
    import numpy as np
    from paper_2609_16575_gb300 import gbpic

    lam0 = 299792458.0 / 9e9
    a, b, L = 0.03 / lam0, 0.015 / lam0, 1.0 / lam0
    om = 2 * np.pi
    beta_c = np.sqrt(om ** 2 - (np.pi / a) ** 2)
    vg = beta_c / om
    rows = []
    for na, nb, nl, nt, paper_eps in WAVEGUIDE_GRIDS[:count]:
        n = (nl - 1, na - 1, nb - 1)
        d = (L / n[0], a / n[1], b / n[2])
        dt = 0.5 / np.sqrt(sum(1.0 / v ** 2 for v in d))
        ctx = gbpic.Context(n, d, dt, precision=gbpic.PIC_FP64 if fp64 else gbpic.PIC_FP32, bc_x=1)
        ctx.set_pec(1, 1)
        ctx.set_port(1.0, om, 2.0, 1)
        ms, _ = time_steps(ctx, torch, nt)
        E, _, _ = ctx.get_fields()
        ctx.close()
        t_end = nt * dt
        j = n[1] // 2
        x = np.arange(n[0] + 1) * d[0]
        x_hi = vg * (t_end - 20.0)          # the envelope has risen to 1 - exp(-10) behind here
        sel = (x >= L / 16) & (x <= x_hi)
        f = E[2, n[2] // 2, j, sel]
        A, beta = _fit_wave(x[sel], f, beta_c)
        A_ref = np.sin(np.pi * j * d[1] / a)
        rows.append({"nodes": [na, nb, nl], "cells": list(n), "steps": nt, "dh": float(np.sqrt(sum(v * v for v in d)) * lam0),
                     "eps_amplitude": abs(A - A_ref) / A_ref, "eps_beta": abs(beta - beta_c) / beta_c,
                     "paper_eps_E0": paper_eps, "cell_updates_per_s": n[0] * n[1] * n[2] * nt / (ms / 1e3),
                     "fit_wavelengths": float((x_hi - L / 16))})
    out = {"workload": "TE10 waveguide a = 3 cm, b = 1.5 cm, L = 1 m, 9 GHz, Courant 0.5, "
                       + ("FP64" if fp64 else "FP32"), "grids": rows}
    if len(rows) >= 3:
        lh = np.log([r["dh"] for r in rows])
        for key in ("eps_amplitude", "eps_beta"):
            out[key + "_rate"] = float(np.polyfit(lh, np.log([r[key] for r in rows]), 1)[0])
    return out


def adjoint_cost(torch, steps=200, precisions=("f64", "f32")):
    """Backward/forward cost of the checkpointed adjoint on the differentiable-run
    workload (32^3, 16 per cell, u_th = 0.02, plane wave of amplitude 0.05, 200 steps,
    checkpoints every 20), on the FP64 and the FP32 path."""
    import numpy as np
    from paper_2609_16575_gb300 import gbpic
    from paper_2609_16575_gb300 import workloads as W

    wl = W.differentiable()
    n, d = wl.n, wl.d
    # a vacuum plane wave along x polarised in y: E_y = cos(k x), B_z = cos(k x') one half
    # step earlier at the B location (an input shape only)
    k = 2 * np.pi / (n[0] * d[0])
    x_e = np.arange(n[0]) * d[0]
    x_b = (np.arange(n[0]) + 0.5) * d[0]
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    E[1] = np.cos(k * x_e)[None, None, :]
    B[2] = np.cos(k * (x_b + 0.5 * wl.dt))[None, None, :]
    A = 0.05
    s = wl.species[0]
    out = {"workload": f"32^3, 16 ppc, u_th=0.02, plane wave A=0.05, {steps} steps, checkpoint every 20"}
    for prec, name in ((gbpic.PIC_FP64, "f64"), (gbpic.PIC_FP32, "f32")):
        if name not in precisions:
            continue
        def fresh():
            c = gbpic.Context(n, d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True)
            c.set_fields(A * E, A * B)
            c.load_species_array(s.q, s.m, s.P, True)
            torch.cuda.synchronize()
            return c
        # warm-up: the first launch of each kernel loads it
        ctx = fresh()
        ctx.step(2)
        ctx.adjoint_forward(4, 2)
        ctx.adjoint_backward(E, B)
        ctx.close()
        ctx = fresh()
        t0 = time.perf_counter()
        ctx.step(steps)
        ctx.sync()
        t_plain = time.perf_counter() - t0
        ctx.close()
        ctx = fresh()
        t0 = time.perf_counter()
        ctx.adjoint_forward(steps, 20)
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        ctx.adjoint_backward(E, B)
        t_bwd = time.perf_counter() - t0
        ctx.close()
        out[name] = {"forward_plain_s": t_plain, "forward_with_checkpoints_s": t_fwd, "backward_s": t_bwd,
                     "backward_over_forward": t_bwd / t_plain}
    return out


def arm_config(spec, world):
    """The workload description both arms print."""
    n = spec["n"]
    npart = n[0] * n[1] * n[2] * spec["ppc"]
    return {"workload": describe(spec), "cells": n[0] * n[1] * n[2], "particles_per_gpu": npart,
            "precision": "fp32 bulk (the fp64 path on the same inputs under 'fp64'), fp64 reductions",
            "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 (particle SoA {npart * 32 * 2 / 1e9:.1f} GB per GPU, double-buffered)"}


# Yee bytes per cell and step the method must move (FP32): read E, B and J, write E and
# B, clear J = 72 B.  The implementation moves 156 B: two Faraday half steps (read E, B;
# write B: 36 B each) and Ampere (read E, B and the 64-bit fixed-point J; write E; clear
# J: 84 B).
YEE_BYTES_PER_CELL = 72
YEE_IMPL_BYTES_PER_CELL = 2 * 36 + 84


def yee_line(kt, ncell, peak):
    """Yee cell updates per second from the CUDA-event times of the field kernels, with
    the HBM fraction of the method's 72 B per cell."""
    fl, fms = kt.get("faraday_half", (0, 0.0))
    al, ams = kt.get("ampere", (0, 0.0))
    if not al or not fl:
        return None
    per_step_s = (fms / fl * 2 + ams / al) / 1e3
    gbs = YEE_BYTES_PER_CELL * ncell / per_step_s / 1e9
    return {"cell_updates_per_s": ncell / per_step_s, "ms_per_step": per_step_s * 1e3,
            "bytes_per_cell": YEE_BYTES_PER_CELL, "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
            "implementation_bytes_per_cell": YEE_IMPL_BYTES_PER_CELL,
            "note": "three kernels per step (two Faraday half steps and Ampere with the J clear)"}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host's cores (one
    process per core); each step is one oracle cycle of every process over its own 32^3
    sample of the headline workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    spec = workload_spec(args)
    cores = host_cores()
    value, wall, npart = oracle_rate(cores, spec, 32, args.warmup, args.steps)
    sample = (f"per step: one FP64 oracle cycle in each of {cores} processes (one per host core, nproc = {cores}), "
              f"each on its own thermal 32^3 x {spec['ppc']} ppc sample ({npart:,} particles), u_th={spec['u_th']}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(spec, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_rate(ms, npart, steps, dist):
    """Whole-job rate of N independent replicas: the slowest rank's time (max over ranks)
    and all ranks' particle-steps over it.  Returns (max ms, particle-steps/s)."""
    import torch

    world = 1
    if dist is not None:
        world = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, npart * world * steps / (ms / 1e3)


def timed_steps(ctx, torch, steps, dist):
    ctx.set_timing(True)
    ctx.kernel_times()
    l0 = ctx.launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    ctx.step(steps)
    b.record(s)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = a.elapsed_time(b)
    launches = ctx.launch_count() - l0
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    ctx.sync()
    return ms, launches, kt


# FP64 tile kernel: FP64 operations the method needs per particle-step (2 DFMA + DADD +
# DMUL thread instructions, counted by ncu on the thermal workload with the kernel that
# evaluated only the deposit branch each particle needs: 1.584e9 DFMA, 1.338e9 DADD,
# 0.803e9 DMUL for 16,777,216 particles; the branch-free kernel executes 369.8 per
# particle, the extra ones discarded), and the FP64 peak of a GB300 from its unit counts
# and clock: 2 FP64 FMA per clock per SM x 152 SMs x 2.07 GHz x 2 operations.
FP64_OPS_PER_PARTICLE = 316.5
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12


def fp64_alu_roofline(kt, n_particles, peak=None, peak_kind=None):
    """FP64 operations per launch of the FP64 tile kernel over its average launch time,
    against `peak` TFLOP/s (default: the unit-count figure above)."""
    if peak is None:
        peak, peak_kind = FP64_PEAK_TFLOPS, "derived: 2 DFMA/clock/SM x 152 SMs x 2.07 GHz"
    launches, ms = kt["tile_push"]
    avg_s = ms / max(launches, 1) / 1e3
    achieved = FP64_OPS_PER_PARTICLE * n_particles / avg_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "kernel": "k_tile_push<double>", "peak_kind": peak_kind,
            "ops_per_particle": FP64_OPS_PER_PARTICLE}


def measured_fp64_peak(gbpic, dev):
    """TFLOP/s of the library's FP64 FMA probe (8 independent DFMA chains per thread,
    every SM busy), or None."""
    try:
        return gbpic.probe_fp64_rate(dev) / 1e12
    except Exception:
        return None


def roofline(kt, dtype, n_particles, ncell, peak, peak_kind, traffic):
    launches, ms = kt["tile_push"]
    avg_s = ms / max(launches, 1) / 1e3
    algo = PART_BYTES[dtype] * n_particles + TILE_GRID_BYTES[dtype] * ncell
    achieved = algo / avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_tile_push", "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "algorithmic_bytes_per_launch": algo, "avg_launch_ms": avg_s * 1e3}


def energy(d):
    return d["U_E"] + d["U_B"] + d["K_half"]


def run_gbpic(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2609_16575_gb300 import gbpic
    from paper_2609_16575_gb300 import workloads as W

    spec = workload_spec(args)
    n, d, ppc = spec["n"], (spec["d"],) * 3, spec["ppc"]
    ncell = n[0] * n[1] * n[2]
    peak, peak_kind = peaks()
    dev = torch.cuda.current_device()
    # this rank's inputs, drawn on the device; both precisions and the end-to-end run
    # start from them
    X, U, w, dt = W.thermal_device(torch, n, spec["d"], ppc, spec["u_th"], spec["seed"] + rank)
    npart = int(w.shape[0])

    def variant(c):
        if args.deposit == "esirkepov":
            c.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV)
        if args.shape == "tsc":
            c.set_shape(gbpic.PIC_SHAPE_TSC)

    # --- FP32, inputs resident in HBM
    ctx = gbpic.Context(n, d, dt, precision=gbpic.PIC_FP32, rho_ion=1.0, device=dev)
    variant(ctx)
    ctx.load_species(-1.0, 1.0, X, U, w, True)
    d0 = ctx.diagnostics()
    ctx.step(args.warmup)
    ctx.sync()
    with Clocks(dev) as clk:
        ms, launches, kt = timed_steps(ctx, torch, args.steps, dist)
    clocks = clk.summary()
    d1 = ctx.diagnostics()
    ctx.close()
    del ctx
    if d1["n_alive"] != npart:
        raise RuntimeError(f"particles lost: {d1['n_alive']} of {npart}")
    ms_all, value = replica_rate(ms, npart, args.steps, dist)
    traffic = committed_traffic("tile_push", spec["name"], npart)
    rl = roofline(kt, "f32", npart, ncell, peak, peak_kind, traffic)
    step_bytes = PART_BYTES["f32"] + STEP_GRID_BYTES["f32"] / ppc
    f32_checks = {"cycles": args.warmup + args.steps, "energy_rel_change": (energy(d1) - energy(d0)) / energy(d0),
                  "gauss_change_max": d1["gauss_change_max"], "rho_max": d1["rho_max"]}

    # --- FP64 GPU path on the same inputs
    fp64 = None
    if not args.no_fp64:
        k64 = max(3, args.steps // 4)
        ctx = gbpic.Context(n, d, dt, precision=gbpic.PIC_FP64, rho_ion=1.0, device=dev)
        variant(ctx)
        ctx.load_species(-1.0, 1.0, X, U, w, True)
        e0 = ctx.diagnostics()
        ctx.step(2)
        ctx.sync()
        ms64, _, kt64 = timed_steps(ctx, torch, k64, dist)
        e1 = ctx.diagnostics()
        ctx.close()
        del ctx
        if e1["n_alive"] != npart:
            raise RuntimeError(f"FP64 path lost particles: {e1['n_alive']} of {npart}")
        ms64, v64 = replica_rate(ms64, npart, k64, dist)
        fpk = measured_fp64_peak(gbpic, dev)
        fp64 = {"value": v64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                "roofline": roofline(kt64, "f64", npart, ncell, peak, peak_kind, None),
                "alu_roofline": fp64_alu_roofline(
                    kt64, npart, *((fpk, "measured: the library's DFMA probe (pic_probe_fp64_rate) on this GPU")
                                   if fpk else (None, None))),
                "step_hbm_frac": v64 / world * (PART_BYTES["f64"] + STEP_GRID_BYTES["f64"] / ppc) / 1e9 / peak,
                "kernels": kernel_table(kt64),
                "checks": {"cycles": 2 + k64, "energy_rel_change": (energy(e1) - energy(e0)) / energy(e0),
                           "gauss_change_max": e1["gauss_change_max"]}}

    # --- end to end through the public API: the FP64 particle arrays from pinned host
    # memory into a new context, the steps, the FP64 diagnostics back to the host
    e2e = None
    if not args.no_e2e:
        # the pinned host copy of a rank's inputs is 56 B per particle (30 GB at 256^3 x
        # 32); ranks take turns when all of them at once would not fit the host's memory
        need = 56 * npart
        turns = world > 1 and world * need > 0.6 * host_memory_available()

        def run_e2e():
            host = [torch.empty(t.shape, dtype=torch.float64, pin_memory=True) for t in (X, U, w)]
            for h, t in zip(host, (X, U, w)):
                h.copy_(t)
            torch.cuda.synchronize()
            Xh, Uh, wh = (h.numpy() for h in host)
            # the library allocates through torch's caching allocator: start it from the
            # state of a fresh process (its cache of the earlier runs' blocks released)
            torch.cuda.empty_cache()
            if dist is not None and not turns:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = gbpic.Context(n, d, dt, precision=gbpic.PIC_FP32, rho_ion=1.0, device=dev)
            variant(ctx)
            t1 = time.perf_counter()
            ctx.load_species(-1.0, 1.0, Xh, Uh, wh, True)   # returns once the sort is done
            t2 = time.perf_counter()
            ctx.step(args.steps)
            d_e2e = ctx.diagnostics()
            t_run = time.perf_counter() - t0
            ctx.close()
            del host, Xh, Uh, wh
            return t_run, {"context_s": t1 - t0, "load_s": t2 - t1, "steps_and_diagnostics_s": t_run - (t2 - t0)}, \
                d_e2e["n_alive"] == npart

        if turns:
            for r in range(world):
                dist.barrier()
                if r == rank:
                    t_e2e, phases, ok = run_e2e()
            dist.barrier()
        else:
            t_e2e, phases, ok = run_e2e()
        del X, U, w
        torch.cuda.empty_cache()
        if dist is not None:
            t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        ntile = (n[0] // 8) * (n[1] // 8) * (n[2] // 8)
        # particle arrays + the loader's per-tile tables up; its histogram, counters and
        # the diagnostics down
        h2d = 7 * 8 * npart + 4 * ntile * 512 + 12 * ntile
        d2h = 4 * ntile * 512 + 8 * 8 + 4 * ntile + ctypes.sizeof(gbpic.pic_diag)
        e2e = {"value": npart * world * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "seconds": t_e2e,
               "includes": "context creation, H2D of the FP64 particle arrays from pinned host memory, tile sort, "
                           f"{args.steps} steps, FP64 diagnostics and their D2H (bytes per step = per run / steps)",
               "check_n_alive": ok, "phases": phases}
        if turns:
            e2e["note"] = ("ranks ran one after another (their pinned inputs together exceed the host's memory); "
                           "value = all ranks' particle-steps over the slowest rank's time")
    else:
        del X, U, w
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec)
    extra, adj = None, None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = other_workloads(torch, peak, peak_kind)
        adj = adjoint_cost(torch)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(arm_config(spec, world), **({"variant": f"deposit={args.deposit}, shape={args.shape}"}
                                                            if args.deposit != "zigzag" or args.shape != "cic" else {})),
                "roofline": rl,
                "step_hbm_frac": value / world * step_bytes / 1e9 / peak,
                "cell_steps_per_s": ncell * world * args.steps / (ms_all / 1e3),
                "yee": yee_line(kt, ncell, peak),
                "kernels": kernel_table(kt), "gpu_launches": launches, "clocks": clocks, "checks": f32_checks,
                "e2e": e2e, "cpu_baseline": cpu, "fp64": fp64, "other_workloads": extra, "adjoint": adj}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.waveguide > 0:
        import torch

        torch.cuda.set_device(0)
        import __graft_entry__

        __graft_entry__.build()
        print(json.dumps(waveguide_convergence(torch, args.waveguide, not args.waveguide_fp32)), flush=True)
        return 0
    if args.adjoint_only > 0:
        import torch

        torch.cuda.set_device(0)
        import __graft_entry__

        __graft_entry__.build()
        precs = ("f32", "f64") if args.adjoint_prec == "both" else (args.adjoint_prec,)
        print(json.dumps(adjoint_cost(torch, args.adjoint_only, precs)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gbpic(args)


if __name__ == "__main__":
    sys.exit(main())
