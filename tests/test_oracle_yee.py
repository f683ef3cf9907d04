"""Pins of the oracle's Yee field solver (section 2.3, Eqs. (13)-(14)) against the
exact discrete vacuum eigenmodes and the divergence identities."""
import numpy as np
import pytest

import oracle


def _run_vacuum(n, d, dt, E, B, steps):
    F = oracle.empty_fields(n)
    F[0:3] = E
    F[3:6] = B
    oracle.run(n, d, dt, F, [], steps)
    return F


@pytest.mark.parametrize("mode,e_hat", [
    ((1, 0, 0), (0, 1, 0)),          # +x wave, Ey / Bz
    ((0, 0, 2), (1, 0, 0)),          # +z wave, Ex / By
    ((1, 2, 0), None),               # oblique in x-y, Ez / Bx, By
    ((1, -1, 2), None),              # fully 3D, generic polarisation
])
def test_yee_plane_wave_is_exact_eigenmode(mode, e_hat):
    """The Yee dispersion relation (sin(w dt/2)/dt)^2 = sum (sin(k d/2)/d)^2 holds
    exactly: a discrete plane wave advances by the closed-form phase to round-off."""
    n = (6, 8, 10)
    d = (0.3, 0.25, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    k = 2 * np.pi * np.array(mode) / (np.array(n) * np.array(d))
    kappa = 2 / np.array(d) * np.sin(k * np.array(d) / 2)
    if e_hat is None:
        # any vector orthogonal to kappa
        e_hat = np.cross(kappa, [0.3, 0.5, 0.9])
        e_hat /= np.linalg.norm(e_hat)
    E0, B0, w = oracle.plane_wave(n, d, dt, mode, e_hat, 0.7)
    steps = 37
    F = _run_vacuum(n, d, dt, E0, B0, steps)
    E1, B1, _ = oracle.plane_wave(n, d, dt, mode, e_hat, 0.7, t_e=steps * dt)
    assert np.abs(F[0:3] - E1).max() < 1e-12
    assert np.abs(F[3:6] - B1).max() < 1e-12
    # a wrong frequency would show up immediately: the continuum w = |k| is off
    assert abs(w - np.linalg.norm(k)) > 1e-4


def test_yee_divergence_identities():
    """div B stays zero and div E stays constant in vacuum (discrete div curl = 0)."""
    rng = np.random.default_rng(7)
    n = (5, 6, 7)
    d = (0.2, 0.3, 0.25)
    dt = oracle.courant_dt(d, 0.5)
    F = oracle.empty_fields(n)
    F[0:3] = rng.standard_normal(F[0:3].shape)
    div_e0 = oracle.divergence(n, d, F[0:3])
    oracle.run(n, d, dt, F, [], 25)
    assert np.abs(oracle.divergence_b(n, d, F[3:6])).max() < 1e-12
    assert np.abs(oracle.divergence(n, d, F[0:3]) - div_e0).max() < 1e-11


def test_yee_faraday_sign_and_staggering():
    """Bx update of Eq. (13) on a hand-sized case: Ez varying along y only."""
    n = (2, 4, 2)
    d = (1.0, 0.5, 1.0)
    dt = 0.1
    E = np.zeros((3, 2, 4, 2))
    E[2, :, :, :] = np.array([0.0, 1.0, 3.0, 6.0])[None, :, None]    # Ez(j)
    B = np.zeros((3, 2, 4, 2))
    oracle.faraday(n, d, dt, E, B, 1.0)
    # Bx(j+1/2) = -dt/dy (Ez(j+1) - Ez(j)), periodic in j
    expect = -dt / 0.5 * (np.roll([0.0, 1.0, 3.0, 6.0], -1) - np.array([0.0, 1.0, 3.0, 6.0]))
    assert np.allclose(B[0, 0, :, 0], expect, atol=1e-15)
    assert np.abs(B[1:]).max() == 0.0


def test_courant_step():
    """Eq. (15): dt at Courant 0.5 of the 3D CFL limit."""
    assert abs(oracle.courant_dt((0.1, 0.1, 0.1)) - 0.5 * 0.1 / np.sqrt(3)) < 1e-17
