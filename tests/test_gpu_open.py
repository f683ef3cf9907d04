"""GPU parity of the open x boundaries (absorbing Mur faces, the soft laser sheet and
particle removal; the boundary and external-source modules of section 2.6 as the
laser-wakefield run of section 4 uses them) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, oracle_n, prepare, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _vacuum_pulse(n=(40, 8, 8), d=(0.1, 0.12, 0.15)):
    """Ey and Ez pulses centred in x, modulated in y and z, in an open-x vacuum box."""
    dt = oracle.courant_dt(d, 0.5)
    nx = n[0]
    x = np.arange(nx + 1)
    y = np.arange(n[1])
    z = np.arange(n[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    E = np.zeros((3, n[2], n[1], nx + 1))
    E[1] = np.exp(-((X - nx / 2) / 2.5) ** 2) * (1 + 0.3 * np.cos(2 * np.pi * Z / n[2]))
    E[2] = 0.5 * np.exp(-((X - nx / 2 - 3) / 3.0) ** 2) * (1 + 0.2 * np.sin(2 * np.pi * Y / n[1]))
    wl = W.Workload("pulse", n, d, dt, 0.0, [], E, None, bc_x=1)
    return wl


def _chunks(wl, prec, chunks):
    """Step the library and the oracle side by side; yield after every chunk."""
    ctx = run_gpu(wl, prec, 0)
    F, osp, _ = run_oracle(wl, prec, 0)
    laser = None if wl.laser is None else wl.laser.as_tuple()
    done = 0
    for k in chunks:
        ctx.step(k)
        ctx.sync()
        oracle.run(oracle_n(wl), wl.d, wl.dt, F, osp, k, step0=done, laser=laser)
        done += k
        yield ctx, F, osp, done


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_mur_faces_vacuum_pulse(prec):
    """Pulses that reach and leave through both faces: every field array, including the
    face plane x = n, follows the oracle, and almost nothing is reflected."""
    wl = _vacuum_pulse()
    tol = 2e-6 if prec == FP32 else 1e-12
    scale = np.abs(wl.E).max()
    e0 = None
    for ctx, F, _, done in _chunks(wl, prec, (30, 30, 100)):
        E, B, J = ctx.get_fields()
        assert E.shape == F[0:3].shape
        errE = np.abs(E - F[0:3]).max() / scale
        errB = np.abs(B - F[3:6]).max() / scale
        assert errE <= tol and errB <= tol, (done, errE, errB)
        assert np.abs(J).max() == 0.0
        if e0 is None:
            e0 = (F[0:6] ** 2).sum()
    # what stays after 160 steps is the 3D Mur residue of the modulated parts
    assert (F[0:6] ** 2).sum() < 3e-2 * e0


def _mini_lwfa():
    wl = W.lwfa(n=(48, 16, 16), ppc_per_dim=2, density=0.05, x0=8, ramp=12, a0=2.0, w0_lambda=1.0,
                fwhm_periods=1.0, plane=2)
    wl.laser.t_peak = 1.5 * wl.laser.tau
    return wl


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_laser_sheet_into_plasma(prec):
    """A relativistic (a0 = 2) pulse launched by the sheet, entering a density ramp:
    fields, currents and every electron follow the oracle over 110 cycles."""
    wl = _mini_lwfa()
    tol_f = 2e-4 if prec == FP32 else 1e-10
    for ctx, F, osp, done in _chunks(wl, prec, (40, 70)):
        E, B, J = ctx.get_fields()
        assert rel_err(E, F[0:3]) <= tol_f, (done, "E", rel_err(E, F[0:3]))
        assert rel_err(B, F[3:6]) <= tol_f, (done, "B", rel_err(B, F[3:6]))
        # the library stores no J on the face plane x = n (the face E follows the Mur
        # condition, so no update reads it); the oracle's Jy, Jz there are left out
        assert np.abs(J[..., -1]).max() == 0.0
        assert rel_err(J[..., :-1], F[6:9, ..., :-1]) <= tol_f, (done, "J", rel_err(J[..., :-1], F[6:9, ..., :-1]))
        P = ctx.get_particles(0)
        Q = osp[0].P
        assert P.shape == Q.shape
        assert np.abs(P[0:3] - Q[0:3]).max() <= (1e-4 if prec == FP32 else 1e-11)
        assert rel_err(P[3:6], Q[3:6]) <= tol_f, (done, "u", rel_err(P[3:6], Q[3:6]))
    assert np.abs(Q[3:6]).max() > 0.1      # the pulse did reach the electrons


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_particles_leave_through_faces(prec):
    """A hot plasma in a short open box: particles leave through both faces, the
    library drops exactly the ones the oracle zeroes, counts them, and the survivors
    match."""
    wl = W.thermal((16, 8, 8), 0.2, 4, 0.6, seed=61)
    wl.bc_x = 1
    wl.rho_ion = 0.0
    ctx = run_gpu(wl, prec, 12)
    F, osp, _ = run_oracle(wl, prec, 12)
    P = ctx.get_particles(0)
    Q = osp[0].P
    gone_gpu = np.isnan(P[6])
    gone_or = Q[6] == 0.0
    assert gone_or.sum() > 50
    assert np.array_equal(gone_gpu, gone_or)
    assert ctx.diagnostics()["n_escaped"] == gone_or.sum()
    assert ctx.diagnostics()["n_alive"] == (~gone_or).sum()
    keep = ~gone_or
    tol = 2e-5 if prec == FP32 else 1e-11
    assert np.abs(P[0:3, keep] - Q[0:3, keep]).max() <= tol * 10
    assert rel_err(P[3:6, keep], Q[3:6, keep]) <= tol
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol
    assert rel_err(B, F[3:6]) <= tol


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_beam_spills_and_exits(prec):
    """A fast beam filling tiles that held nothing at load: the receiving tiles overflow,
    the overflow is pushed from the spill list, and the beam leaves through x = n."""
    n, d = (16, 8, 8), (0.2, 0.2, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    rng = np.random.Generator(np.random.PCG64(62))
    npart = 3000
    P = np.empty((7, npart))
    P[0] = rng.random(npart) * 6.0
    P[1] = rng.random(npart) * n[1]
    P[2] = rng.random(npart) * n[2]
    P[3] = 3.0 + 0.1 * rng.standard_normal(npart)
    P[4] = 0.05 * rng.standard_normal(npart)
    P[5] = 0.05 * rng.standard_normal(npart)
    P[6] = 1e-4
    wl = W.Workload("beam", n, d, dt, 0.0, [W.SpeciesInput(-1.0, 1.0, P)], bc_x=1)
    ctx = run_gpu(wl, prec, 45)
    F, osp, _ = run_oracle(wl, prec, 45)
    Pg = ctx.get_particles(0)
    Q = osp[0].P
    gone_or = Q[6] == 0.0
    assert npart // 4 < gone_or.sum() < npart * 3 // 4
    assert np.array_equal(np.isnan(Pg[6]), gone_or)
    keep = ~gone_or
    tol = 1e-4 if prec == FP32 else 1e-10
    assert np.abs(Pg[0:3, keep] - Q[0:3, keep]).max() <= tol
    assert rel_err(Pg[3:6, keep], Q[3:6, keep]) <= tol
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])


def test_open_x_argument_checks():
    """The laser needs an open x and a plane inside the box; fields must have n + 1
    values per x line."""
    from paper_2609_16575_gb300 import gbpic
    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=0)
    with pytest.raises(gbpic.PicError):
        c.set_laser(1.0, 1.0, 1.0, 1.0, 1.0, 4, 4.0, 4.0)
    c.close()
    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=1)
    with pytest.raises(gbpic.PicError):
        c.set_laser(1.0, 1.0, 1.0, 1.0, 1.0, 16, 4.0, 4.0)
    with pytest.raises(ValueError):
        c.set_fields(np.zeros((3, 8, 8, 16)), None)
    c.set_laser(1.0, 1.0, 1.0, 1.0, 1.0, 3, 4.0, 4.0)
    c.close()
