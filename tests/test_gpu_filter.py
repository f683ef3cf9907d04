"""GPU parity of the compensated binomial current filter (section 2.2 "compensated
smoothing", section 2.6 current filtering; the scheme is a reading of those passages) against
the FP64 oracle, on a periodic thermal plasma and on the open-x laser wakefield with a
moving window."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, oracle_n, prepare, rel_err

pytestmark = pytest.mark.gpu


def _pair(wl, prec, filt, window=None):
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True, bc_x=wl.bc_x)
    ctx.set_current_filter(*filt)
    if wl.laser is not None:
        ctx.set_laser(*wl.laser.as_tuple())
    if window is not None:
        ctx.set_moving_window(window["start"], window["every"], window["species"], window["ppc"],
                              window["density"], window["x0"], window["ramp"])
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    F = oracle.empty_fields(oracle_n(wl))
    if E is not None:
        F[0:3] = E
    if B is not None:
        F[3:6] = B
    osp = [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]
    return ctx, F, osp


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("filt", [(1, 1), (2, 0), (3, 1)])
def test_filtered_thermal_plasma(prec, filt):
    """A hot periodic plasma (grid 24 x 16 x 8, u_th = 0.3) for 12 filtered cycles:
    fields, the filtered J and every particle follow the oracle."""
    wl = W.thermal((24, 16, 8), 0.2, 4, 0.3, seed=91)
    ctx, F, osp = _pair(wl, prec, filt)
    ctx.step(12)
    ctx.sync()
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 12, current_filter=filt)
    tol = 2e-5 if prec == FP32 else 1e-11
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])
    assert rel_err(J, F[6:9]) <= tol, rel_err(J, F[6:9])
    P = ctx.get_particles(0)
    Q = osp[0].P
    d = P[0:3] - Q[0:3]
    for k in range(3):
        d[k] = (d[k] + wl.n[k] / 2) % wl.n[k] - wl.n[k] / 2
    assert np.abs(d).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert rel_err(P[3:6], Q[3:6]) <= tol
    # the filter broke the discrete continuity equation, as it must
    dg = ctx.diagnostics()
    ctx.step(1)
    dg = ctx.diagnostics()
    assert dg["cont_max"] > 1e-6 * dg["J_max"] / min(wl.d)
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_filtered_laser_wakefield_with_window(prec):
    """The mini laser wakefield with the filter (2 passes, compensated) and a moving window:
    the open x is filtered with zero outside the box; 40 cycles against the oracle."""
    wl = W.lwfa(n=(48, 16, 16), ppc_per_dim=2, density=0.05, x0=8, ramp=12, a0=2.0, w0_lambda=1.0,
                fwhm_periods=1.0, plane=2)
    wl.laser.t_peak = 1.5 * wl.laser.tau
    win = dict(start=10, every=int(math.ceil(wl.d[0] / wl.dt)), species=0, ppc=(2, 2, 2), density=0.05, x0=8.0,
               ramp=12.0)
    filt = (2, 1)
    ctx, F, osp = _pair(wl, prec, filt, window=win)
    ctx.step(40)
    ctx.sync()
    oracle.run_window(oracle_n(wl), wl.d, wl.dt, F, osp, 40, win, laser=wl.laser.as_tuple(), current_filter=filt)
    tol = 2e-4 if prec == FP32 else 1e-10
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])
    assert rel_err(J[..., :-1], F[6:9, ..., :-1]) <= tol
    P = ctx.get_particles(0)
    Q = osp[0].P
    gone = Q[6] == 0.0
    assert np.array_equal(np.isnan(P[6]), gone)
    keep = ~gone
    assert np.abs(P[0:3, keep] - Q[0:3, keep]).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert rel_err(P[3:6, keep], Q[3:6, keep]) <= tol
    ctx.close()


def test_filter_argument_checks():
    from paper_2609_16575_gb300 import gbpic

    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, track_ids=True)
    for bad in ((-1, 1), (9, 1), (1, 2)):
        with pytest.raises(gbpic.PicError):
            c.set_current_filter(*bad)
    c.set_current_filter(1, 1)
    c.load_species_array(-1.0, 1.0, np.array([[1.5], [1.5], [1.5], [0.1], [0.0], [0.0], [1e-3]]), True)
    with pytest.raises(gbpic.PicError):
        c.adjoint_forward(4, 2)            # the adjoint has no filter
    c.set_current_filter(0)
    c.step(2)
    c.sync()
    c.close()
