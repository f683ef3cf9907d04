"""GPU parity of the moving window (section 2.2: an operation at the end of the cycle;
section 4: the laser-wakefield run moves its window along the pulse) against the FP64
oracle: fields, every particle (the loaded ones, the ones the window removed and the
plasma it brought in) and the counters, over many moves."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, oracle_n, prepare, rel_err

pytestmark = pytest.mark.gpu


def _mini_lwfa(n=(48, 16, 16)):
    wl = W.lwfa(n=n, ppc_per_dim=2, density=0.05, x0=8, ramp=12, a0=2.0, w0_lambda=1.0, fwhm_periods=1.0, plane=2)
    wl.laser.t_peak = 1.5 * wl.laser.tau
    return wl


def _window(wl, start):
    return dict(start=start, every=int(math.ceil(wl.d[0] / wl.dt)), species=0, ppc=(2, 2, 2), density=0.05,
                x0=8.0, ramp=12.0)


def _gpu(wl, prec, win):
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=0.0, track_ids=True, bc_x=1)
    ctx.set_laser(*wl.laser.as_tuple())
    ctx.set_moving_window(win["start"], win["every"], win["species"], win["ppc"], win["density"], win["x0"],
                          win["ramp"])
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    return ctx


def _oracle(wl, prec):
    sp, E, B = prepare(wl, prec)
    F = oracle.empty_fields(oracle_n(wl))
    osp = [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]
    return F, osp


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_window_follows_the_oracle(prec):
    """A relativistic pulse driven into a density ramp while the window moves every 3
    cycles from cycle 20 on: 60 cycles, 13 moves.  Fields, the last J, every electron
    (removed ones read as NaN) and the removal count follow the oracle."""
    wl = _mini_lwfa()
    win = _window(wl, 20)
    assert win["every"] == 3
    ctx = _gpu(wl, prec, win)
    F, osp = _oracle(wl, prec)
    n0 = osp[0].n
    laser = wl.laser.as_tuple()
    tol_f = 2e-4 if prec == FP32 else 1e-10
    done = 0
    for k in (25, 35):
        ctx.step(k)
        ctx.sync()
        oracle.run_window(oracle_n(wl), wl.d, wl.dt, F, osp, k, win, step0=done, laser=laser)
        done += k
        assert ctx.window_moves() == oracle.window_moves_before(win, done)
        E, B, J = ctx.get_fields()
        assert rel_err(E, F[0:3]) <= tol_f, (done, "E", rel_err(E, F[0:3]))
        assert rel_err(B, F[3:6]) <= tol_f, (done, "B", rel_err(B, F[3:6]))
        # no J is stored on the face plane x = n (its face E follows the Mur condition)
        assert rel_err(J[..., :-1], F[6:9, ..., :-1]) <= tol_f, (done, "J")
        P = ctx.get_particles(0)
        Q = osp[0].P
        assert P.shape == Q.shape, (P.shape, Q.shape)
        gone = Q[6] == 0.0
        assert np.array_equal(np.isnan(P[6]), gone)
        keep = ~gone
        assert np.abs(P[0:3, keep] - Q[0:3, keep]).max() <= (1e-4 if prec == FP32 else 1e-11)
        assert rel_err(P[3:6, keep], Q[3:6, keep]) <= tol_f, (done, "u")
        assert rel_err(P[6, keep], Q[6, keep]) <= (1e-7 if prec == FP32 else 0.0)
        d = ctx.diagnostics()
        assert d["n_escaped"] == gone.sum()
        assert d["n_alive"] == keep.sum()
    assert ctx.window_moves() == 13
    assert osp[0].n > n0 and gone[:n0].sum() > 0          # plasma came in and left
    assert np.abs(Q[3:6, keep]).max() > 0.1                # the pulse reached the electrons
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_window_with_esirkepov(prec):
    """Esirkepov's deposit under the moving window: the crossers' records are exported in
    the cycles that end with a move (every stored x cell drops by one) like in the
    others; 30 cycles from the first move on, fields, J and every electron against the
    oracle."""
    from paper_2609_16575_gb300 import gbpic

    wl = _mini_lwfa()
    win = _window(wl, 0)
    ctx = _gpu(wl, prec, win)
    ctx.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV)
    F, osp = _oracle(wl, prec)
    ctx.step(30)
    oracle.run_window(oracle_n(wl), wl.d, wl.dt, F, osp, 30, win, laser=wl.laser.as_tuple(), guide={"esirkepov": 1})
    assert ctx.window_moves() == oracle.window_moves_before(win, 30) == 10
    tol_f = 2e-4 if prec == FP32 else 1e-10
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol_f, ("E", rel_err(E, F[0:3]))
    assert rel_err(B, F[3:6]) <= tol_f, ("B", rel_err(B, F[3:6]))
    assert rel_err(J[..., :-1], F[6:9, ..., :-1]) <= tol_f, "J"
    P = ctx.get_particles(0)
    Q = osp[0].P
    assert P.shape == Q.shape, (P.shape, Q.shape)
    gone = Q[6] == 0.0
    assert np.array_equal(np.isnan(P[6]), gone)
    keep = ~gone
    assert np.abs(P[0:3, keep] - Q[0:3, keep]).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert rel_err(P[3:6, keep], Q[3:6, keep]) <= tol_f
    ctx.close()


def test_window_plasma_fills_empty_tiles():
    """A window that starts over vacuum and moves every cycle into a plateau: after 40
    moves the whole front of the window holds the plateau lattice at rest, with the
    weights and the count the profile gives, and nothing spilled."""
    from paper_2609_16575_gb300 import gbpic

    n, d = (32, 8, 8), (0.2, 0.2, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    ctx = gbpic.Context(n, d, dt, precision=FP32, rho_ion=0.0, track_ids=False, bc_x=1)
    ctx.set_moving_window(0, 1, 0, (2, 1, 2), 0.8, 36.0, 0.0)
    ctx.load_species_array(-1.0, 1.0, np.zeros((7, 0)), True)
    ctx.step(40)
    ctx.sync()
    P = ctx.get_particles(0)
    # absolute x of the window's cell 0 is 40: plasma from x = 36, i.e. window cells 0..31
    assert P.shape[1] == 32 * 8 * 8 * 4
    assert np.all(P[3:6] == 0.0)
    np.testing.assert_allclose(P[6], 0.8 * 0.008 / 4, rtol=1e-7)
    xs = np.sort(np.unique(np.round(P[0] % 1.0, 6)))
    np.testing.assert_array_equal(xs, [0.25, 0.75])
    dg = ctx.diagnostics()
    assert dg["n_spilled"] == 0 and dg["n_escaped"] == 4 * 8 * 8 * 4
    ctx.close()


def test_window_argument_checks():
    """The window needs an open x, valid numbers, and must precede loading its species
    and stepping."""
    from paper_2609_16575_gb300 import gbpic

    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=0)
    with pytest.raises(gbpic.PicError):
        c.set_moving_window(0, 1, 0, (1, 1, 1), 1.0, 0.0, 0.0)
    c.close()
    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=1)
    for bad in ((0, 0, 0, (1, 1, 1), 1.0, 0.0, 0.0), (0, 1, 0, (0, 1, 1), 1.0, 0.0, 0.0),
                (0, 1, 0, (1, 1, 1), -1.0, 0.0, 0.0), (0, 1, 0, (65, 1, 1), 1.0, 0.0, 0.0),
                (0, 1, 0, (1, 1, 1), 1.0, 0.0, -2.0)):
        with pytest.raises(gbpic.PicError):
            c.set_moving_window(*bad)
    c.load_species_array(-1.0, 1.0, np.array([[1.5], [1.5], [1.5], [0.0], [0.0], [0.0], [1e-3]]), True)
    with pytest.raises(gbpic.PicError):
        c.set_moving_window(0, 1, 0, (1, 1, 1), 1.0, 0.0, 0.0)      # species 0 already loaded
    c.set_moving_window(0, 1, 1, (1, 1, 1), 1.0, 0.0, 0.0)
    with pytest.raises(gbpic.PicError):
        c.step(1)                                                   # species 1 not loaded
    c.close()
