"""Checkpoint / resume through pic_save_state / pic_load_state: a run stopped, saved,
restored into a fresh context and continued equals the run that never stopped, up to the
rounding of the current's partial sums (they follow the particles' order in the tiles,
which the restore sorts again): the FP32 and FP64 tolerances of the parity tests."""
import math

import numpy as np
import pytest

from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, prepare

pytestmark = pytest.mark.gpu


def _new(wl, prec, window=None):
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True, bc_x=wl.bc_x)
    if wl.laser is not None:
        ctx.set_laser(*wl.laser.as_tuple())
    if window is not None:
        ctx.set_moving_window(*window)
    return ctx


def _load(ctx, wl, prec):
    sp, E, B = prepare(wl, prec)
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)


def _compare(a, b, prec):
    tol = 2e-5 if prec == FP32 else 1e-12
    Ea, Ba, Ja = a.get_fields()
    Eb, Bb, Jb = b.get_fields()
    Pa, Pb = a.get_particles(0), b.get_particles(0)
    assert Pa.shape == Pb.shape
    assert np.abs(Ea - Eb).max() <= tol * np.abs(Ea).max()
    assert np.abs(Ba - Bb).max() <= tol * np.abs(Ba).max()
    assert np.abs(Ja - Jb).max() <= tol * np.abs(Ja).max()
    assert np.array_equal(np.isnan(Pa), np.isnan(Pb))
    keep = ~np.isnan(Pa[6])
    assert np.abs(Pa[0:3, keep] - Pb[0:3, keep]).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert np.abs(Pa[3:7, keep] - Pb[3:7, keep]).max() <= tol * np.abs(Pa[3:6, keep]).max()
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("step", "n_alive", "n_escaped"):
        assert da[k] == db[k], k


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_resume_thermal(prec):
    wl = W.thermal((24, 16, 8), 0.2, 4, 0.3, seed=131)
    a = _new(wl, prec)
    _load(a, wl, prec)
    a.step(20)
    b = _new(wl, prec)
    _load(b, wl, prec)
    b.step(10)
    blob = b.save_state()
    b.close()
    c = _new(wl, prec)
    c.load_state(blob)
    assert c.diagnostics()["step"] == 10
    c.step(10)
    _compare(a, c, prec)
    a.close()
    c.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_resume_laser_wakefield_with_window(prec):
    """Open x, the laser sheet, particles leaving and a moving window bringing plasma in:
    the move count, the injected ids and the escape count carry over."""
    wl = W.lwfa(n=(48, 16, 16), ppc_per_dim=2, density=0.05, x0=8, ramp=12, a0=2.0, w0_lambda=1.0,
                fwhm_periods=1.0, plane=2)
    wl.laser.t_peak = 1.5 * wl.laser.tau
    window = (5, int(math.ceil(wl.d[0] / wl.dt)), 0, (2, 2, 2), 0.05, 8.0, 12.0)
    a = _new(wl, prec, window)
    _load(a, wl, prec)
    a.step(40)
    b = _new(wl, prec, window)
    _load(b, wl, prec)
    b.step(21)
    blob = b.save_state()
    b.close()
    c = _new(wl, prec, window)
    c.load_state(blob)
    assert c.window_moves() == 5        # moves after cycles 7, 10, 13, 16, 19
    c.step(19)
    assert c.window_moves() == a.window_moves() == 11   # ... 22, 25, ..., 37
    _compare(a, c, prec)
    a.close()
    c.close()


def test_state_argument_checks():
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.1, seed=132)
    a = _new(wl, FP32)
    _load(a, wl, FP32)
    a.step(2)
    blob = a.save_state()
    other = gbpic.Context((16, 8, 16), wl.d, wl.dt, precision=FP32, track_ids=True)
    with pytest.raises(gbpic.PicError):
        other.load_state(blob)                       # another grid
    other.close()
    with pytest.raises(gbpic.PicError):
        a.load_state(blob)                           # not a fresh context
    fresh = _new(wl, FP32)
    with pytest.raises(gbpic.PicError):
        fresh.load_state(blob[:-8])                  # truncated
    fresh.load_state(blob)
    assert fresh.diagnostics()["n_alive"] == a.diagnostics()["n_alive"]
    a.close()
    fresh.close()


def test_diagnostics_log(tmp_path):
    """The JSON-lines log: one record per call, non-finite values written as null."""
    import json

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.1, seed=133)
    a = _new(wl, FP32)
    _load(a, wl, FP32)
    path = tmp_path / "diag.jsonl"
    a.log_diagnostics(path, run="t")
    a.step(1)
    a.log_diagnostics(path, run="t")
    recs = [json.loads(line) for line in open(path)]
    assert [r["step"] for r in recs] == [0, 1]
    assert recs[0]["cont_max"] is None and recs[1]["cont_max"] is not None
    assert recs[1]["n_alive"] == wl.species[0].P.shape[1] and recs[1]["run"] == "t"
    a.close()
