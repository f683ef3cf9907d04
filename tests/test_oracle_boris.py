"""Pins of the oracle's relativistic Boris pusher (section 2.4) against closed forms
and the numbers printed in section 3.1."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _circle_radius(pts):
    # algebraic (Kasa) least-squares circle fit
    A = np.c_[2 * pts[:, 0], 2 * pts[:, 1], np.ones(len(pts))]
    b = (pts ** 2).sum(1)
    cx, cy, c = np.linalg.lstsq(A, b, rcond=None)[0]
    return math.sqrt(c + cx * cx + cy * cy)


def test_boris_pure_B_larmor_convergence():
    """Section 3.1, pure-B benchmark: the orbit's radius equals the closed form
    R = (v/Omega) sqrt(1 + (Omega dt/2)^2) of the Boris rotation, and its error
    converges with the slope the paper prints (1.998)."""
    g = GOLD["boris_B_points_per_period"]
    v = g["v_y"]
    gam = 1.0 / math.sqrt(1 - v * v)
    errs, dts = [], []
    for npt in g["value"]:
        dt = 2 * math.pi * gam / (npt - 1)
        xs, us = oracle.boris_orbit([0, 0, 0], [0, 0, 1], -1.0, dt, [0, 0, 0], [0, v * gam, 0],
                                    g["periods"] * (npt - 1), backpush=True)
        R = _circle_radius(xs[-(npt - 1):, :2])
        rL = v * gam
        closed = math.sqrt(1 + (math.pi / (npt - 1)) ** 2) - 1
        assert abs((R / rL - 1) - closed) < 1e-9
        gam_run = np.sqrt(1 + (us ** 2).sum(1))
        assert np.abs(gam_run / gam - 1).max() < 1e-12     # paper: ~1e-15 per step
        errs.append(R / rL - 1)
        dts.append(dt)
    slope, icpt = np.polyfit(np.log(dts), np.log(errs), 1)
    fit = slope * np.log(dts) + icpt
    r2 = 1 - np.sum((np.log(errs) - fit) ** 2) / np.sum((np.log(errs) - np.mean(np.log(errs))) ** 2)
    assert abs(slope - GOLD["boris_B_larmor_slope"]["value"]) < 0.005
    assert r2 > 0.9999


def test_boris_rotation_phase_closed_form():
    """Pure B: u turns by exactly theta = 2 atan(Omega dt / 2) per step (with the
    sense of rotation of q B), so after N steps the phase is N theta."""
    gam = 3.0
    u0 = np.array([math.sqrt(gam ** 2 - 1), 0.0, 0.0])
    B = 0.7
    dt = 0.37
    N = 10000
    xs, us = oracle.boris_orbit([0, 0, 0], [0, 0, B], -1.0, dt, [0, 0, 0], u0, N, backpush=False)
    Omega = B / gam
    theta = 2 * math.atan(Omega * dt / 2)
    # an electron (q < 0) in B = +z gyrates counter-clockwise
    phase = math.atan2(us[-1, 1], us[-1, 0])
    expect = math.remainder(N * theta, 2 * math.pi)
    assert abs(math.remainder(phase - expect, 2 * math.pi)) < 1e-11
    assert abs(np.linalg.norm(us[-1]) / np.linalg.norm(u0) - 1) < 1e-13


def test_boris_pure_E_second_order():
    """Section 3.1, pure-E benchmark: with the half back-push the momentum is the
    exact midpoint value u^{n+1/2} = (q/m) E (n+1/2) dt, the position at t = 1
    converges with the paper's slope (2.002) to x = -(sqrt(1+t^2) - 1), and equals
    a brute-force midpoint sum of the exact velocity."""
    errs, dts = [], []
    for N in GOLD["boris_E_samples"]["value"]:
        dt = 1.0 / (N - 1)
        xs, us = oracle.boris_orbit([1, 0, 0], [0, 0, 0], -1.0, dt, [0, 0, 0], [0, 0, 0], N - 1, backpush=True)
        u_exact = -(N - 1.5) * dt
        assert abs(us[-1, 0] - u_exact) / abs(u_exact) < GOLD["boris_E_velocity_error_max"]["value"] * 10
        mids = (np.arange(N - 1) + 0.5) * dt
        brute = math.fsum(-dt * m / math.sqrt(1 + m * m) for m in mids)
        assert abs(xs[-1, 0] - brute) < 1e-12
        x_exact = -(math.sqrt(2.0) - 1)
        errs.append(abs(xs[-1, 0] - x_exact) / abs(x_exact))
        dts.append(dt)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - GOLD["boris_E_position_slope"]["value"]) < 0.005


def test_boris_without_backpush_is_first_order():
    """The reading that momenta start half a step behind (u^{-1/2}) is what gives the
    paper's second-order pure-E convergence: starting from u^{-1/2} = 0 instead
    loses an order."""
    errs, dts = [], []
    for N in [101, 201, 401, 801]:
        dt = 1.0 / (N - 1)
        xs, _ = oracle.boris_orbit([1, 0, 0], [0, 0, 0], -1.0, dt, [0, 0, 0], [0, 0, 0], N - 1, backpush=False)
        x_exact = -(math.sqrt(2.0) - 1)
        errs.append(abs(xs[-1, 0] - x_exact))
        dts.append(dt)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - 1.0) < 0.05


def test_boris_exb_drift_fixed_point():
    """E x B drift: with E = E0 y and B = B0 z the Boris map has the fixed point
    u = U x with U / sqrt(1 + U^2 + (eps E0)^2) = E0 / B0 (eps = q dt / 2m), so a
    particle started there keeps u to round-off and moves at
    v = (E0/B0) sqrt(1 + U^2 + (eps E0)^2) / sqrt(1 + U^2), i.e. the drift
    E x B / B^2 up to (eps E0)^2 / 2."""
    E0, B0, dt, q = 0.05, 1.0, 0.1, -1.0
    eps = q * dt / 2
    r = E0 / B0
    # U^2 (1 - r^2) = r^2 (1 + (eps E0)^2)
    U = r * math.sqrt((1 + (eps * E0) ** 2) / (1 - r * r))
    xs, us = oracle.boris_orbit([0, E0, 0], [0, 0, B0], q, dt, [0, 0, 0], [U, 0, 0], 2000, backpush=False)
    assert np.abs(us - us[0]).max() < 1e-14
    v = (xs[-1, 0] - xs[0, 0]) / (2000 * dt)
    assert abs(v / (U / math.sqrt(1 + U * U)) - 1) < 1e-12
    assert abs(v / r - 1) < (eps * E0) ** 2           # E x B / B^2 within the Boris offset
    assert abs(xs[-1, 1]) < 1e-12 and abs(xs[-1, 2]) < 1e-12


def test_boris_exb_gyroaverage_from_rest():
    """A particle released from rest in crossed fields (|E| << |B|) drifts on average
    at E x B / B^2 (the relativistic corrections are O((E/B)^2))."""
    E0, B0, dt = 1e-4, 1.0, 0.05
    gam_period = 2 * math.pi / B0
    steps_per = int(round(gam_period / dt))
    nper = 50
    xs, us = oracle.boris_orbit([0, E0, 0], [0, 0, B0], -1.0, dt, [0, 0, 0], [0, 0, 0], steps_per * nper, backpush=True)
    # the Boris gyro period is 2 pi / theta steps; average over whole turns of the discrete orbit
    theta = 2 * math.atan(B0 * dt / 2)
    nturn_steps = int(round(nper * 2 * math.pi / theta))
    v = xs[nturn_steps, 0] / (nturn_steps * dt)
    assert abs(v / (E0 / B0) - 1) < 2e-3
