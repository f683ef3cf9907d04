"""Helpers shared by the GPU parity tests: run one seeded input through the CUDA
library (via the C ABI binding) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2609_16575_gb300 import workloads as W

FP32, FP64 = 0, 1


def quantize_fields(E, precision):
    if E is None:
        return None
    return E.astype(np.float32).astype(np.float64) if precision == FP32 else E.copy()


def prepare(wl: W.Workload, precision: int):
    """Inputs as the working precision can hold them (both sides get these)."""
    sp = []
    for s in wl.species:
        P = W.quantize_fp32(s.P) if precision == FP32 else s.P.copy()
        sp.append(W.SpeciesInput(s.q, s.m, P, s.momenta_at_half_step))
    return sp, quantize_fields(wl.E, precision), quantize_fields(wl.B, precision)


def run_gpu(wl: W.Workload, precision: int, steps: int, track_ids=True, record_every=0, slack=0.0, per_step=None):
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, precision)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=precision, rho_ion=wl.rho_ion, track_ids=track_ids,
                        record_every=record_every, bc_x=wl.bc_x)
    if wl.laser is not None:
        ctx.set_laser(*wl.laser.as_tuple())
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step, capacity_slack=slack)
    if per_step is None:
        ctx.step(steps)
    else:
        for k in range(steps):
            per_step(ctx, k)
            ctx.step(1)
    ctx.sync()
    return ctx


def oracle_n(wl: W.Workload):
    """Grid description for the oracle: (nx, ny, nz[, open x])."""
    return tuple(wl.n) + ((1,) if wl.bc_x else ())


def run_oracle(wl: W.Workload, precision: int, steps: int, per_step=None):
    sp, E, B = prepare(wl, precision)
    n = oracle_n(wl)
    laser = None if wl.laser is None else wl.laser.as_tuple()
    F = oracle.empty_fields(n)
    if E is not None:
        F[0:3] = E
    if B is not None:
        F[3:6] = B
    osp = [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]
    for s, si in zip(osp, sp):
        if not si.momenta_at_half_step:
            oracle.backpush(n, wl.d, wl.dt, F[0:3], F[3:6], s)
    hist = []
    if per_step is None:
        if steps:
            hist = oracle.run(n, wl.d, wl.dt, F, osp, steps, laser=laser)
    else:
        for k in range(steps):
            per_step(F, osp, k)
            hist.append(oracle.run(n, wl.d, wl.dt, F, osp, 1, step0=k, laser=laser)[0])
        hist = np.array(hist)
    return F, osp, hist


def rel_err(a, b):
    """Normwise relative error max|a - b| / max|b| (absolute when b is zero)."""
    scale = np.abs(b).max()
    diff = np.abs(a - b).max()
    return diff / scale if scale > 0 else diff


def wrapped_diff(Xa, Xb, n):
    d = Xa - Xb
    for k in range(3):
        d[k] = (d[k] + n[k] / 2) % n[k] - n[k] / 2
    return d


def plane_wave_fields(n, d, dt, amplitude=0.05, modes=(((1, 0, 0), (0, 1, 0)), ((0, 2, 1), None))):
    """A superposition of discrete vacuum eigenmodes as a smooth non-zero initial field."""
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    for mode, e_hat in modes:
        k = 2 * np.pi * np.array(mode) / (np.array(n) * np.array(d))
        kappa = 2 / np.array(d) * np.sin(k * np.array(d) / 2)
        if e_hat is None:
            e_hat = np.cross(kappa, [0.3, 0.5, 0.9])
            e_hat = e_hat / np.linalg.norm(e_hat)
        e, b, _ = oracle.plane_wave(n, d, dt, mode, e_hat, amplitude)
        E += e
        B += b
    return E, B
