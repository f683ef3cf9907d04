"""Pins of the oracle's open x boundaries (absorbing faces with first-order Mur, laser
sheet source, particle removal), the external-source and boundary modules of section
2.6 used by the laser-wakefield setup of section 4."""
import numpy as np

import oracle
from paper_2609_16575_gb300 import workloads as W


def _pulse_energy_left(courant_like_1d):
    nx = 200
    n = (nx, 1, 1, 1)
    dtr = 1e4 if courant_like_1d else 0.1
    d = (0.1, dtr, dtr)
    dt = oracle.courant_dt(d, 0.999999 if courant_like_1d else 0.5)
    F = oracle.empty_fields(n)
    x = np.arange(nx + 1) * 0.1
    F[1, 0, 0, :] = np.exp(-((x - 10.0) / 0.8) ** 2)
    e0 = (F[0:6] ** 2).sum()
    oracle.run(n, d, dt, F, [], int(3 * nx * 0.1 / dt))
    return (F[0:6] ** 2).sum() / e0


def test_mur_absorbs_normal_incidence():
    """A pulse split into two halves leaving through both x faces: first-order Mur is
    exact for normally incident waves of the Yee scheme, so nothing is reflected (at
    the 1D magic time step and at the 3D Courant-0.5 step alike)."""
    assert _pulse_energy_left(True) < 1e-20
    assert _pulse_energy_left(False) < 1e-12


def test_open_box_interior_equals_periodic_box():
    """While nothing reaches the faces, an open-x box evolves exactly like the periodic one
    (the stencils widen the field support by one cell per step: 4 steps from x = 10..14
    stay clear of the faces of a 24-cell box)."""
    wl = W.thermal((24, 6, 6), 0.2, 2, 0.05, seed=51)
    P = wl.species[0].P
    P[0] = 10 + np.mod(P[0], 4)         # particles in the middle of the box
    nP, nO = wl.n, tuple(wl.n) + (1,)
    Fp = oracle.empty_fields(nP)
    Fo = oracle.empty_fields(nO)
    sp_p = [oracle.Species(-1.0, 1.0, P)]
    sp_o = [oracle.Species(-1.0, 1.0, P)]
    oracle.run(nP, wl.d, wl.dt, Fp, sp_p, 4)
    oracle.run(nO, wl.d, wl.dt, Fo, sp_o, 4)
    assert np.abs(Fo[:, :, :, :24] - Fp).max() == 0.0
    assert np.abs(Fo[:, :, :, 24]).max() == 0.0
    assert np.abs(sp_o[0].P - sp_p[0].P).max() == 0.0


def test_laser_sheet_amplitude():
    """The soft sheet J_y = -2 a(t)/dx radiates a field of amplitude a(t) to each side
    (to the discrete-source factor of a few percent at 20 cells per wavelength); the
    backward half is absorbed at x = 0."""
    nx = 400
    lam = 2 * np.pi
    d = (lam / 20, 1e4, 1e4)
    n = (nx, 1, 1, 1)
    dt = oracle.courant_dt(d, 0.5)
    laser = (2.0, 1.0, 1e9, 10 * lam, 40.0, 20, 0.0, 0.0)
    F = oracle.empty_fields(n)
    probe = []
    for s in range(int(150 / dt)):
        oracle.run(n, d, dt, F, [], 1, step0=s, laser=laser)
        probe.append(F[1, 0, 0, 300])
    peak = np.abs(probe).max()
    assert abs(peak / 2.0 - 1) < 0.03
    assert np.abs(F[1, 0, 0, :15]).max() < 0.1 * peak      # only the source tail is left near x = 0


def test_particles_leaving_open_faces_are_removed():
    n = (8, 4, 4, 1)
    d = (0.2, 0.2, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    P = np.array([[7.95, 0.05, 4.0], [1.5, 1.5, 1.5], [1.5, 1.5, 1.5],
                  [0.9, -0.9, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1e-3, 1e-3, 1e-3]])
    sp = [oracle.Species(-1.0, 1.0, P)]
    F = oracle.empty_fields(n)
    oracle.run(n, d, dt, F, sp, 2)
    w = sp[0].P[6]
    assert w[0] == 0.0 and w[1] == 0.0 and w[2] == 1e-3
