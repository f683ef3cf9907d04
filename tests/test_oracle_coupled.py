"""Pins of the oracle's full PIC cycle (section 2.2, Fig. 2) against the paper's
plasma-oscillation benchmark (section 3.3), a closed-form discrete cold-plasma
frequency, Gauss's law preservation and the energy history."""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import least_squares

import oracle
from paper_2609_16575_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _prepare(wl, gauss=False):
    n, d = wl.n, wl.d
    sp = [oracle.Species(s.q, s.m, s.P.copy()) for s in wl.species]
    F = oracle.empty_fields(n)
    if gauss:
        E, worst = oracle.gauss_x(n, d, oracle.rho(n, d, sp, wl.rho_ion))
        assert worst < 1e-14
        F[0:3] = E
    for s, si in zip(sp, wl.species):
        if not si.momenta_at_half_step:
            oracle.backpush(n, d, wl.dt, F[0:3], F[3:6], s)
    return F, sp


def _fit_omega(t, y, guess=1.0):
    r = least_squares(lambda p: p[0] * np.cos(p[1] * t + p[2]) + p[3] - y,
                      [np.abs(y).max(), guess, 0.0, 0.0], xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return r.x[1]


def test_paper_plasma_oscillation():
    """Section 3.3: 2 x 2 x 100 cells over L = 2 pi, C = 0.5, v_z = 1e-3 sin z.
    The E_z probe at z = L/4 oscillates at w/w_p = 1 (paper) and, more sharply, at the
    closed-form discrete frequency; U_EM + K varies by less than 7.5e-4 (paper);
    the continuity residual of the last step is ~1e-13 (paper)."""
    wl = W.paper_cold_plasma(steps=2000)
    n, d = wl.n, wl.d
    F, sp = _prepare(wl)
    probe, hist = [], []
    for s in range(wl.steps):
        probe.append(F[2][n[2] // 4].mean())
        if s == wl.steps - 1:
            r0 = oracle.rho(n, d, sp, wl.rho_ion)
        hist.append(oracle.run(n, d, wl.dt, F, sp, 1)[0])
    r1 = oracle.rho(n, d, sp, wl.rho_ion)
    t = np.arange(wl.steps) * wl.dt
    w = _fit_omega(t, np.array(probe))
    assert abs(w - GOLD["cold_plasma_omega"]["value"]) < 1e-3
    assert abs(w - oracle.cold_plasma_omega(2 * np.pi / 100, wl.dt)) < 1e-6
    U = np.array(hist).sum(1)
    assert (U.max() - U.min()) / U.mean() < GOLD["cold_plasma_energy_variation"]["value"]
    R = oracle.continuity_residual(n, d, wl.dt, r0, r1, F[6:9])
    assert np.abs(R).max() * min(d) < 10 * GOLD["cold_plasma_continuity_residual"]["value"]


def test_cold_plasma_cube_frequency():
    """Cold-plasma workload (16^3, dx = 0.1, 8 per cell, FP64, 200 steps): the k = 2 pi/L
    mode of Ex oscillates at w_eff = sqrt(1 - sin^2(k dx/2)/2) corrected for leapfrog."""
    wl = W.cold_plasma()
    n, d = wl.n, wl.d
    F, sp = _prepare(wl, gauss=True)
    amps = []
    for s in range(wl.steps):
        amps.append(np.fft.rfft(F[0].mean(axis=(0, 1)))[1])
        oracle.run(n, d, wl.dt, F, sp, 1)
    a = np.array(amps)
    y = a.imag if np.abs(a.imag).max() > np.abs(a.real).max() else a.real
    w = _fit_omega(np.arange(wl.steps) * wl.dt, y)
    w_closed = oracle.cold_plasma_omega(2 * np.pi / 16, wl.dt)
    assert abs(w / w_closed - 1) < 1e-5
    assert abs(w_closed - 0.99047) < 1e-5


def test_gauss_law_preserved_thermal():
    """Gauss's law (2) stays as it started (G^n - G^0 = 0) when particles move in all
    three dimensions and cross cells: the deposit is charge conserving and the Yee
    update keeps div E - rho constant (section 2.3)."""
    wl = W.thermal((6, 5, 4), 0.2, 8, 0.3, seed=5, steps=15)
    n, d = wl.n, wl.d
    F, sp = _prepare(wl)
    G0 = oracle.divergence(n, d, F[0:3]) - oracle.rho(n, d, sp, wl.rho_ion)
    for _ in range(wl.steps):
        r_before = oracle.rho(n, d, sp, wl.rho_ion)
        oracle.run(n, d, wl.dt, F, sp, 1)
        r_after = oracle.rho(n, d, sp, wl.rho_ion)
        R = oracle.continuity_residual(n, d, wl.dt, r_before, r_after, F[6:9])
        assert np.abs(R).max() * wl.dt < 1e-13 * (np.abs(r_before).max() + 1)
    G = oracle.divergence(n, d, F[0:3]) - oracle.rho(n, d, sp, wl.rho_ion)
    assert np.abs(G - G0).max() < 1e-12 * np.abs(G0).max()


def test_energy_history_levels():
    """The energy diagnostic is U_E(E^n), U_B(B^n) with B^n the average of Eq. (21),
    and K with gamma^n = (gamma^{n-1/2} + gamma^{n+1/2})/2: checked against the
    same sums written out with numpy on one step of a small thermal state."""
    wl = W.thermal((4, 4, 4), 0.2, 4, 0.2, seed=9)
    n, d, dt = wl.n, wl.d, wl.dt
    rng = np.random.default_rng(3)
    F = oracle.empty_fields(n)
    F[0:6] = rng.standard_normal(F[0:6].shape) * 0.1
    sp = [oracle.Species(s.q, s.m, s.P.copy()) for s in wl.species]
    E0 = F[0:3].copy()
    Bhalf = F[3:6].copy()
    u0 = sp[0].P[3:6].copy()
    h = oracle.run(n, d, dt, F, sp, 1)[0]
    Bn = Bhalf.copy()
    oracle.faraday(n, d, dt, E0, Bn, 0.5)
    dV = np.prod(d)
    assert abs(h[0] - 0.5 * dV * (E0 ** 2).sum()) < 1e-13
    assert abs(h[1] / (0.5 * dV * (Bn ** 2).sum()) - 1) < 1e-12
    g0 = np.sqrt(1 + (u0 ** 2).sum(0))
    g1 = np.sqrt(1 + (sp[0].P[3:6] ** 2).sum(0))
    K = (sp[0].P[6] * (0.5 * (g0 + g1) - 1)).sum()
    assert abs(h[2] / K - 1) < 1e-12
