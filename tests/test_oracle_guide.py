"""Pins of the oracle's perfectly conducting walls and waveguide port (section 3.2: the
Yee solver is verified on the TE10 mode of a perfectly conducting rectangular guide
driven at its input plane).

The discrete TE_m0 mode of a guide of width a = n_y dy is an exact eigenvector of the
Yee scheme: E_z = A sin(k_y y) sin(k_x x - w t) with k_y = m pi / a, the magnetic field
from Faraday's law, and the discrete dispersion relation
(2/dt sin(w dt/2))^2 = (2/dx sin(k_x dx/2))^2 + (2/dy sin(k_y dy/2))^2."""
import numpy as np

import oracle


def _kappa(k, h):
    return 2.0 / h * np.sin(k * h / 2.0)


def _te_mode(n, d, dt, mode_x, mode_y, amplitude=1.0):
    """E (at t = 0) and B (at t = -dt/2) of the discrete TE_{mode_y,0} mode travelling
    along +x with mode_x wavelengths in the periodic x length; E along z."""
    nx, ny, nz = n
    kx = 2 * np.pi * mode_x / (nx * d[0])
    ky = np.pi * mode_y / (ny * d[1])
    kapx, kapy = _kappa(kx, d[0]), _kappa(ky, d[1])
    Om = np.sqrt(kapx ** 2 + kapy ** 2)
    w = 2.0 / dt * np.arcsin(Om * dt / 2.0)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y = ii * d[0], jj * d[1]
    E = np.zeros((3, nz, ny, nx))
    B = np.zeros((3, nz, ny, nx))
    t_b = -dt / 2
    E[2] = amplitude * np.sin(ky * y) * np.sin(kx * x)
    # Bx at (i, j + 1/2, k + 1/2), By at (i + 1/2, j, k + 1/2)
    B[0] = -amplitude * kapy / Om * np.cos(ky * (y + d[1] / 2)) * np.cos(kx * x - w * t_b)
    B[1] = -amplitude * kapx / Om * np.sin(ky * y) * np.sin(kx * (x + d[0] / 2) - w * t_b)
    return E, B, w, kx, ky


def test_te10_is_an_exact_mode_of_the_conducting_guide():
    """A periodic-x box with the wall plane y = 0 (and z = 0) conducting: the TE10 mode
    (half a wave across the guide) comes back after 300 steps exactly as the closed form
    says, while without the wall the same field does not stay a mode."""
    n, d = (16, 12, 3), (0.1, 0.13, 0.1)
    dt = oracle.courant_dt(d, 0.5)
    E, B, w, kx, ky = _te_mode(n, d, dt, 2, 1)
    steps = 300
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    ref = np.sin(ky * jj * d[1]) * np.sin(kx * ii * d[0] - w * steps * dt)
    for pec, expect_exact in ((dict(pec_y=1, pec_z=1), True), (None, False)):
        F = oracle.empty_fields(n)
        F[0:3], F[3:6] = E, B
        oracle.run(n, d, dt, F, [], steps, guide=pec)
        err = np.abs(F[2] - ref).max()
        if expect_exact:
            assert err < 1e-11, err
            assert np.abs(F[0:2]).max() < 1e-13 and np.abs(F[2, :, 0, :]).max() == 0.0
        else:
            assert err > 1e-2, err


def test_port_launches_the_te10_mode():
    """The hard port on x = 0 of an open guide (walls y = 0, z = 0; width 18 cells of
    lambda / 20) at 1.11 times the cut-off: after the envelope has risen, the field
    downstream has the port's amplitude and the discrete mode's propagation constant,
    and its transverse profile is the half sine."""
    dx = 1.0 / 20
    nx, ny, nz = 240, 18, 1
    d = (dx, dx, dx)
    dt = oracle.courant_dt(d, 0.5)
    om = 2 * np.pi
    guide = dict(pec_y=1, pec_z=1, port=1, e0=1.0, omega=om, tau=1.0, mode_y=1)
    n = (nx, ny, nz, 1)
    F = oracle.empty_fields(n)
    steps = int(12 / dt)
    probes = [(20, 9), (40, 9), (40, 3)]
    rec = []
    for s in range(steps):
        oracle.run(n, d, dt, F, [], 1, step0=s, guide=guide)
        rec.append([F[2, 0, j, i] for i, j in probes])
    rec = np.array(rec)
    t = (np.arange(steps) + 1) * dt
    late = t > 8.0
    A = np.stack([np.sin(om * t[late]), np.cos(om * t[late])], 1)
    fits = [np.linalg.lstsq(A, rec[late, q], rcond=None)[0] for q in range(3)]
    amp = [np.hypot(*c) for c in fits]
    ph = [np.arctan2(c[1], c[0]) for c in fits]
    assert abs(amp[0] - 1.0) < 2e-3 and abs(amp[1] - 1.0) < 2e-3, amp
    np.testing.assert_allclose(amp[2] / amp[1], np.sin(np.pi * 3 / ny), rtol=2e-3)
    ky = np.pi / (ny * dx)
    Om = 2 / dt * np.sin(om * dt / 2)
    beta = 2 / dx * np.arcsin(np.sqrt(Om ** 2 - _kappa(ky, dx) ** 2) * dx / 2)
    beta_fit = np.mod(ph[0] - ph[1], 2 * np.pi) / (20 * dx)      # 20 cells: one free-space wavelength
    np.testing.assert_allclose(beta_fit, beta, rtol=1e-3)
    assert np.abs(F[2, :, 0, :]).max() == 0.0                     # the wall
    assert beta < om                                               # a guided (slow) wave
