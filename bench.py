#!/usr/bin/env python
"""Benchmark of the GB300 explicit EM-PIC hot path (KEMPIC-3D cycle: Faraday half
step, fused gather + Boris + zigzag deposit, Faraday half step, Ampere).

Workload: thermal plasma, 128^3 periodic cells, dx = 0.2 c/w_p, 64 electrons per
cell (134,217,728 particles) at uniform random positions with Maxwellian momenta
u_th = 0.05 c, immobile ions, dt = 0.5 x Courant, FP32 bulk.  One step = one full
PIC cycle over every particle and cell.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbpic|reference]

Under torchrun every rank runs its own replica (the method has no exchange step on
one GPU; replicas only) and the value is the sum over ranks of particle-steps
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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
WORKLOAD = dict(n=(128, 128, 128), d=0.2, ppc=64, u_th=0.05, seed=1235)
# algorithmic bytes (what the method must move; sorting, ghosts and the fixed-point
# width of J are overheads counted against the achieved fraction)
PART_BYTES = {"f32": 60, "f64": 112}       # read cell + 3 offsets + 3 momenta + w, write all but w
TILE_GRID_BYTES = {"f32": 36, "f64": 72}   # gather reads E, B (24 B) + deposit writes J (12 B) per cell
STEP_GRID_BYTES = {"f32": 108, "f64": 216}  # + Yee: read E, B, J, write E, B, zero J (72 B)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gbpic", choices=["gbpic", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the other workloads and the adjoint cost")
    p.add_argument("--adjoint-only", type=int, default=0,
                   help="only time the FP64 checkpointed adjoint of the differentiable run over this many steps")
    p.add_argument("--stress", type=int, default=0,
                   help="also run the 256^3 x 32 ppc precision-stress workload for this many steps (FP32 and FP64)")
    p.add_argument("--waveguide", type=int, default=0,
                   help="run the first N grids of the TE10 waveguide convergence study (FP64) and exit")
    p.add_argument("--waveguide-fp32", action="store_true", help="the waveguide study on the FP32 path")
    p.add_argument("--small", action="store_true", help="32^3 cells instead of 128^3 (smoke)")
    p.add_argument("--cells", type=int, default=0, help="cells per dimension (profiling cases); 0 = 128")
    p.add_argument("--sort-every", type=int, default=0, help="tile re-sort cadence passed to the library")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("push.cu", "pic_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2609_16575_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
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


def make_workload(small, rank, cells=0):
    from paper_2609_16575_gb300 import workloads as W

    n = (32, 32, 32) if small else (cells,) * 3 if cells else WORKLOAD["n"]
    return W.thermal(n, WORKLOAD["d"], WORKLOAD["ppc"], WORKLOAD["u_th"], seed=WORKLOAD["seed"] + rank)


def cpu_baseline(steps=10, n=32):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload shape:
    a 32^3-cell box at 64 per cell (2.1M particles), `steps` cycles, one host core."""
    import oracle
    from paper_2609_16575_gb300 import workloads as W

    wl = W.thermal((n, n, n), WORKLOAD["d"], WORKLOAD["ppc"], WORKLOAD["u_th"], seed=WORKLOAD["seed"])
    sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
    F = oracle.empty_fields(wl.n)
    oracle.run(wl.n, wl.d, wl.dt, F, sp, 1)    # warm (page-in, library load)
    t0 = time.perf_counter()
    oracle.run(wl.n, wl.d, wl.dt, F, sp, steps)
    dt = time.perf_counter() - t0
    npart = wl.nparticles
    return {"value": npart * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"thermal {n}^3 cells x 64 ppc ({npart} particles), {steps} cycles, FP64, single thread",
            "seconds": round(dt, 2)}


def time_steps(ctx, torch, steps):
    """CUDA-event time (ms) of `steps` cycles on the context's stream."""
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.set_timing(True)
    ctx.kernel_times()
    a.record(st)
    ctx.step(steps)
    b.record(st)
    torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.set_timing(False)
    return a.elapsed_time(b), kt


def other_workloads(torch, peak):
    """Throughput on the other workload shapes: the cold-plasma oscillation (16^3, 8 per
    cell, FP64 and FP32) and the laser wakefield (512 x 128 x 128, open x, 8 per cell,
    FP32)."""
    from paper_2609_16575_gb300 import gbpic
    from paper_2609_16575_gb300 import workloads as W

    out = {}
    wl = W.cold_plasma(n=16)
    for prec, name in ((gbpic.PIC_FP64, "f64"), (gbpic.PIC_FP32, "f32")):
        ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion)
        s = wl.species[0]
        ctx.load_species_array(s.q, s.m, s.P, True)
        time_steps(ctx, torch, 5)
        ms, _ = time_steps(ctx, torch, 200)
        out[f"cold_plasma_16_{name}"] = {"value": s.n * 200 / (ms / 1e3), "unit": UNIT, "steps": 200,
                                          "ms_per_step": ms / 200, "particles": s.n,
                                          "note": "launch-bound: 32,768 particles fill 8 tiles"}
        ctx.close()
    wl = W.lwfa()
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion, bc_x=1)
    ctx.set_laser(*wl.laser.as_tuple())
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    time_steps(ctx, torch, 3)
    steps = 20
    ms, kt = time_steps(ctx, torch, steps)
    npart = s.n
    ncell = wl.n[0] * wl.n[1] * wl.n[2]
    tl, tms = kt["tile_push"]
    algo = PART_BYTES["f32"] * npart + TILE_GRID_BYTES["f32"] * ncell
    achieved = algo / (tms / tl / 1e3) / 1e9
    out["lwfa_512x128x128_f32"] = {"value": npart * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                                   "ms_per_step": ms / steps, "particles": npart,
                                   "tile_push": {"avg_launch_ms": tms / tl, "achieved_gbs": achieved,
                                                 "frac": achieved / peak},
                                   "yee": yee_line(kt, ncell, peak),
                                   "note": "steps 4-23 of the run: the pulse has not reached the plasma yet"}
    ctx.close()
    # the thermal workload with the compensated binomial current filter (1 pass per
    # dimension and the compensator): the cost of the three filter passes per cycle
    wl = W.thermal((128, 128, 128), WORKLOAD["d"], WORKLOAD["ppc"], WORKLOAD["u_th"], seed=WORKLOAD["seed"])
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion)
    ctx.set_current_filter(1, True)
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, True)
    del wl
    time_steps(ctx, torch, 3)
    steps = 10
    ms, kt = time_steps(ctx, torch, steps)
    out["thermal_128_filtered_f32"] = {
        "value": s.n * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "particles": s.n, "filter": "1 binomial pass + compensator per dimension",
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items() if v[0]},
        "note": "'other' holds the filter: 3 passes over J (3 x 8 bytes read and written per cell each)"}
    ctx.close()
    # the thermal workload with Esirkepov's deposit (the crossers' currents from their
    # 3x3x3 supports, computed by the whole warp)
    wl = W.thermal((128, 128, 128), WORKLOAD["d"], WORKLOAD["ppc"], WORKLOAD["u_th"], seed=WORKLOAD["seed"])
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion)
    ctx.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV)
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, True)
    del wl
    time_steps(ctx, torch, 3)
    steps = 10
    ms, kt = time_steps(ctx, torch, steps)
    out["thermal_128_esirkepov_f32"] = {
        "value": s.n * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "particles": s.n, "deposit": "Esirkepov (CIC)",
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items() if v[0]}}
    ctx.close()
    # the same run with the moving window: a one-cell move every ceil(dx / dt) = 3 cycles
    # from the first cycle on, the new column's plasma injected at each move
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
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items() if v[0]},
        "note": "steps 4-33 with a moving window; 'other' holds the field shift, the injection, the "
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


def stress_run(torch, steps):
    """The precision-stress workload: 256^3 periodic cells, 32 electrons per cell
    (536,870,912), u_th = 0.1, dx = 0.2, immobile ions.  Inputs are drawn on the device
    (torch's Philox generator, seed 1238: uniform positions, Gaussian momenta) and loaded
    through device pointers.  FP32 and FP64 paths from the same inputs: throughput,
    relative change of the total energy U_E + U_B + K over `steps` cycles, and the
    largest change of the Gauss residual."""
    from paper_2609_16575_gb300 import gbpic
    from paper_2609_16575_gb300 import workloads as W

    n, ppc, d, u_th = 256, 32, 0.2, 0.1
    npart = n ** 3 * ppc
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1238)
    X = torch.rand((3, npart), generator=gen, device="cuda", dtype=torch.float64) * n
    X.clamp_(max=n * (1 - 2 ** -40))
    U = torch.randn((3, npart), generator=gen, device="cuda", dtype=torch.float64) * u_th
    w = torch.full((npart,), d ** 3 / ppc, device="cuda", dtype=torch.float64)
    dt = W.courant_dt((d, d, d), 0.5)
    out = {"workload": f"256^3 periodic, 32 ppc ({npart:,} electrons), u_th=0.1, dx=0.2, dt=0.5 Courant, "
                       f"{steps} steps, inputs drawn on the device (Philox, seed 1238)"}
    for prec, name in ((gbpic.PIC_FP32, "f32"), (gbpic.PIC_FP64, "f64")):
        ctx = gbpic.Context((n, n, n), (d, d, d), dt, precision=prec, rho_ion=1.0)
        ctx.load_species(-1.0, 1.0, X, U, w, True)
        d0 = ctx.diagnostics()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ctx.step(steps)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        d1 = ctx.diagnostics()
        e0 = d0["U_E"] + d0["U_B"] + d0["K_half"]
        e1 = d1["U_E"] + d1["U_B"] + d1["K_half"]
        out[name] = {"value": npart * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                     "energy_rel_change": (e1 - e0) / e0, "gauss_change_max": d1["gauss_change_max"],
                     "rho_max": d1["rho_max"], "n_alive": d1["n_alive"]}
        ctx.close()
        del ctx
    del X, U, w
    return out


def arm_config(n, npart, ncell, world, sort_every):
    """The workload description both arms print."""
    return {"workload": (f"thermal plasma {n}^3 periodic, dx=0.2, 64 ppc ({npart:,} electrons), "
                         "u_th=0.05, immobile ions, dt=0.5 Courant"),
            "particles_per_gpu": npart, "cells": ncell, "precision": "fp32 bulk, fp64 reductions",
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (particle SoA 4.3 GB per GPU)"}


# Yee kernels per cell and step (FP32): two Faraday half steps (read E, B; write B: 36 B
# each) and Ampere (read E, B and the 64-bit J; write E; clear J: 84 B)
YEE_BYTES_PER_CELL = 2 * 36 + 84


def yee_line(kt, ncell, peak):
    """Yee cell updates per second from the CUDA-event times of the field kernels."""
    fl, fms = kt.get("faraday_half", (0, 0.0))
    al, ams = kt.get("ampere", (0, 0.0))
    if not al or not fl:
        return None
    per_step_s = (fms / fl * 2 + ams / al) / 1e3
    gbs = YEE_BYTES_PER_CELL * ncell / per_step_s / 1e9
    return {"cell_updates_per_s": ncell / per_step_s, "ms_per_step": per_step_s * 1e3,
            "bytes_per_cell": YEE_BYTES_PER_CELL, "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
            "note": "fields (about 105 MB at 128^3) largely stay in the 129 MB L2 between kernels"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    from paper_2609_16575_gb300 import workloads as W

    # each step: one oracle cycle over a 16^3-cell box at 64 per cell (262,144 particles)
    wl = W.thermal((16, 16, 16), WORKLOAD["d"], WORKLOAD["ppc"], WORKLOAD["u_th"], seed=WORKLOAD["seed"])
    sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
    F = oracle.empty_fields(wl.n)
    oracle.run(wl.n, wl.d, wl.dt, F, sp, args.warmup)
    t0 = time.perf_counter()
    oracle.run(wl.n, wl.d, wl.dt, F, sp, args.steps)
    dt = time.perf_counter() - t0
    value = wl.nparticles * args.steps / dt
    sample = f"thermal 16^3 cells x 64 ppc ({wl.nparticles} particles) per step, FP64 oracle, single thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(WORKLOAD["n"][0], WORKLOAD["ppc"] * WORKLOAD["n"][0] ** 3, WORKLOAD["n"][0] ** 3,
                                 args.gpus, args.sort_every),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def fp64_alu_roofline(kt, n_particles):
    launches, ms = kt["tile_push"]
    avg_s = ms / max(launches, 1) / 1e3
    achieved = FP64_OPS_PER_PARTICLE * n_particles / avg_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "kernel": "k_tile_push<double>",
            "peak_kind": "derived: 2 DFMA/clock/SM x 152 SMs x 2.07 GHz (a DFMA probe reached 1.02 TFLOP/s)",
            "ops_per_particle": FP64_OPS_PER_PARTICLE}


def roofline(kt, dtype, n_particles, ncell, peak, peak_kind, traffic):
    launches, ms = kt["tile_push"]
    avg_s = ms / max(launches, 1) / 1e3
    algo = PART_BYTES[dtype] * n_particles + TILE_GRID_BYTES[dtype] * ncell
    achieved = algo / avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_tile_push", "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "algorithmic_bytes_per_launch": algo, "avg_launch_ms": avg_s * 1e3}


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

    wl = make_workload(args.small, rank, args.cells)
    P = wl.species[0].P
    npart = P.shape[1]
    ncell = wl.ncells
    peak, peak_kind = peaks()
    dev = torch.cuda.current_device()

    # --- FP32, inputs resident in HBM
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion, device=dev,
                        sort_every=args.sort_every)
    ctx.set_fields(None, None)
    ctx.load_species_array(-1.0, 1.0, P)
    ctx.step(args.warmup)
    ctx.sync()
    with Clocks(dev) as clk:
        ms, launches, kt = timed_steps(ctx, torch, args.steps, dist)
    clocks = clk.summary()
    diag = ctx.diagnostics()
    ctx.sync()
    if diag["n_alive"] != npart:
        raise RuntimeError(f"particles lost: {diag['n_alive']} of {npart}")
    ctx.close()
    del ctx
    ms_all, value = replica_rate(ms, npart, args.steps, dist)
    wk = f"thermal{wl.n[0]}"
    traffic = committed_traffic("tile_push", wk, npart)
    rl = roofline(kt, "f32", npart, ncell, peak, peak_kind, traffic)
    step_bytes = PART_BYTES["f32"] + STEP_GRID_BYTES["f32"] / WORKLOAD["ppc"]
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items() if v[0]}

    # --- FP64 GPU path on the same workload
    fp64 = None
    if not args.no_fp64:
        k64 = max(3, args.steps // 10)
        ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP64, rho_ion=wl.rho_ion, device=dev)
        ctx.set_fields(None, None)
        ctx.load_species_array(-1.0, 1.0, P)
        ctx.step(2)
        ctx.sync()
        ms64, _, kt64 = timed_steps(ctx, torch, k64, dist)
        ctx.close()
        del ctx
        v64 = npart * k64 / (ms64 / 1e3)
        fp64 = {"value": v64 * world, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                "roofline": roofline(kt64, "f64", npart, ncell, peak, peak_kind, None),
                "alu_roofline": fp64_alu_roofline(kt64, npart),
                "step_hbm_frac": v64 * (PART_BYTES["f64"] + STEP_GRID_BYTES["f64"] / WORKLOAD["ppc"]) / 1e9 / peak}

    # --- end to end through the public API: host (pinned) inputs in, diagnostics out
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(P.shape, dtype=torch.float64, pin_memory=True)
        pinned.numpy()[:] = P
        Ph = pinned.numpy()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP32, rho_ion=wl.rho_ion, device=dev)
        ctx.set_fields(None, None)
        ctx.load_species_array(-1.0, 1.0, Ph)
        ctx.step(args.steps)
        d_e2e = ctx.diagnostics()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        ctx.close()
        del ctx
        if dist is not None:
            t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        ntile = (wl.n[0] // 8) * (wl.n[1] // 8) * (wl.n[2] // 8)
        h2d = 7 * 8 * npart + 4 * ntile * 512 + 12 * ntile
        d2h = 4 * ntile * 512 + 8 * 8 + 4 * ntile
        e2e = {"value": npart * world * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "includes": "context creation, H2D of the FP64 particle arrays from pinned memory, tile sort, "
                           f"{args.steps} steps, FP64 diagnostics and their D2H",
               "check_n_alive": d_e2e["n_alive"] == npart}
        del pinned

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    extra, adj, stress = None, None, None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = other_workloads(torch, peak)
        adj = adjoint_cost(torch)
    if rank == 0 and world == 1 and args.stress > 0:
        stress = stress_run(torch, args.stress)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": arm_config(wl.n[0], npart, ncell, world, args.sort_every),
                "roofline": rl,
                "step_hbm_frac": value / world * step_bytes / 1e9 / peak,
                "cell_steps_per_s": ncell * world * args.steps / (ms_all / 1e3),
                "yee": yee_line(kt, ncell * world, peak),
                "kernels": kernels, "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
                "cpu_baseline": cpu, "fp64": fp64, "other_workloads": extra, "adjoint": adj}
        if stress is not None:
            line["precision_stress"] = stress
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
        print(json.dumps(adjoint_cost(torch, args.adjoint_only, ("f64",))), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gbpic(args)


if __name__ == "__main__":
    sys.exit(main())
