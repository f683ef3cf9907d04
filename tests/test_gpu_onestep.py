"""One cycle of each optional part of the cycle against the FP64 oracle at the parity
tolerances of a single step (max relative error of every field array and of the
particle state <= 1e-5 on the FP32 path, <= 1e-12 on the FP64 path): the compensated
current filter, Esirkepov's deposit, the conducting walls with the waveguide port, and
a cycle that ends with a moving-window move (new plasma injected).  The longer runs of
the other test files check the same parts over tens of cycles at looser bounds, where
trajectories separate; a fault that appears in one step and then washes out would hide
there, not here."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, oracle_n, plane_wave_fields, prepare, rel_err, wrapped_diff

pytestmark = pytest.mark.gpu

TOL = {FP32: 1e-5, FP64: 1e-12}


def _start(wl, prec, setup):
    """The library context and the oracle state on the same inputs."""
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True, bc_x=wl.bc_x)
    setup(ctx)
    if wl.laser is not None:
        ctx.set_laser(*wl.laser.as_tuple())
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    F = oracle.empty_fields(oracle_n(wl))
    if E is not None:
        F[0:3] = E
    if B is not None:
        F[3:6] = B
    return ctx, F, [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]


def _compare(ctx, F, osp, wl, prec, j_face=True):
    E, B, J = ctx.get_fields()
    tol = TOL[prec]
    assert rel_err(E, F[0:3]) <= tol, ("E", rel_err(E, F[0:3]))
    assert rel_err(B, F[3:6]) <= tol, ("B", rel_err(B, F[3:6]))
    if j_face:
        assert rel_err(J, F[6:9]) <= tol, ("J", rel_err(J, F[6:9]))
    else:   # no J is stored on the face plane x = n of an open x
        assert rel_err(J[..., :-1], F[6:9, ..., :-1]) <= tol, ("J", rel_err(J[..., :-1], F[6:9, ..., :-1]))
    if osp:
        P = ctx.get_particles(0)
        Q = osp[0].P
        assert P.shape == Q.shape
        keep = Q[6] != 0.0
        assert np.array_equal(np.isnan(P[6]), ~keep)
        # positions normwise, as the other arrays (max |dX| / max |X|, X in cell units)
        assert np.abs(wrapped_diff(P[0:3, keep], Q[0:3, keep], wl.n)).max() <= tol * max(wl.n)
        assert rel_err(P[3:6, keep], Q[3:6, keep]) <= tol


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("filt", [(1, 1), (3, 0)])
def test_one_filtered_cycle(prec, filt):
    wl = W.thermal((24, 16, 8), 0.2, 4, 0.3, seed=191)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx, F, osp = _start(wl, prec, lambda c: c.set_current_filter(*filt))
    ctx.step(1)
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 1, current_filter=filt)
    _compare(ctx, F, osp, wl, prec)
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_one_esirkepov_cycle(prec):
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((24, 16, 8), 0.2, 4, 0.3, seed=192)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx, F, osp = _start(wl, prec, lambda c: c.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV))
    ctx.step(1)
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 1, guide=dict(esirkepov=1))
    _compare(ctx, F, osp, wl, prec)
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_one_guide_cycle(prec):
    """Walls on y = 0 and z = 0 and the port on the open face x = 0, one cycle from a
    field of two vacuum modes (the port's first value and the walls act at once)."""
    n, d = (40, 12, 6), (0.05, 0.05, 0.05)
    dt = oracle.courant_dt(d, 0.5)
    E, B = plane_wave_fields(n, d, dt)
    # an open x line holds n + 1 nodes: on the face plane x = n only Ey, Ez and Bx exist
    Ef, Bf = E[..., :1].copy(), B[..., :1].copy()
    Ef[0] = 0.0
    Bf[1:3] = 0.0
    E = np.concatenate([E, Ef], axis=-1)
    B = np.concatenate([B, Bf], axis=-1)
    if prec == FP32:
        E, B = E.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context(n, d, dt, precision=prec, bc_x=1)
    ctx.set_pec(1, 1)
    ctx.set_port(1.0, 2 * np.pi, 0.5, 1)
    ctx.set_fields(E, B)
    ctx.step(1)
    F = oracle.empty_fields(n + (1,))
    F[0:3], F[3:6] = E, B
    oracle.run(n + (1,), d, dt, F, [], 1, guide=dict(pec_y=1, pec_z=1, port=1, e0=1.0, omega=2 * np.pi, tau=0.5,
                                                     mode_y=1))
    Eg, Bg, _ = ctx.get_fields()
    assert rel_err(Eg, F[0:3]) <= TOL[prec], rel_err(Eg, F[0:3])
    assert rel_err(Bg, F[3:6]) <= TOL[prec], rel_err(Bg, F[3:6])
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_one_cycle_with_a_window_move(prec):
    """A laser-wakefield box whose window moves at the end of the first cycle: the field
    shift, the removal of the first column and the plasma injected into the last one."""
    wl = W.lwfa(n=(48, 16, 16), ppc_per_dim=2, density=0.05, x0=8, ramp=12, a0=2.0, w0_lambda=1.0,
                fwhm_periods=1.0, plane=2)
    wl.laser.t_peak = 1.5 * wl.laser.tau
    win = dict(start=0, every=1, species=0, ppc=(2, 2, 2), density=0.05, x0=8.0, ramp=12.0)
    ctx, F, osp = _start(wl, prec, lambda c: c.set_moving_window(win["start"], win["every"], win["species"],
                                                                 win["ppc"], win["density"], win["x0"], win["ramp"]))
    ctx.step(1)
    oracle.run_window(oracle_n(wl), wl.d, wl.dt, F, osp, 1, win, laser=wl.laser.as_tuple())
    assert ctx.window_moves() == 1
    _compare(ctx, F, osp, wl, prec, j_face=False)
    ctx.close()
