"""GPU physics parity: the cold-plasma workload against the oracle and the closed-form
discrete frequency, energy history, discrete continuity and Gauss's law on the GPU
path (FP64 reductions of the diagnostics)."""
import numpy as np
import pytest
from scipy.optimize import least_squares

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _cold_plasma():
    wl = W.cold_plasma()
    sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
    wl.E, worst = oracle.gauss_x(wl.n, wl.d, oracle.rho(wl.n, wl.d, sp, wl.rho_ion))
    wl.B = np.zeros_like(wl.E)
    return wl


def _fit(t, y):
    r = least_squares(lambda p: p[0] * np.cos(p[1] * t + p[2]) + p[3] - y, [np.abs(y).max(), 1.0, 0.0, 0.0],
                      xtol=1e-15, ftol=1e-15, gtol=1e-15)
    return r.x[1]


def test_cold_plasma_fp64_against_oracle():
    """Cold-plasma oscillation, 16^3, 8 per cell, FP64, 200 steps: one step within
    1e-12, the Ex mode history within 1e-9, w within 0.5% of the oracle (in fact
    ~1e-7) and of the closed form, energy history within 1%."""
    wl = _cold_plasma()
    ctx1 = run_gpu(wl, FP64, 1)
    F1, _, _ = run_oracle(wl, FP64, 1)
    E, B, J = ctx1.get_fields()
    assert rel_err(E, F1[0:3]) <= 1e-12
    assert rel_err(J, F1[6:9]) <= 1e-12

    amps_g = []
    ctx = run_gpu(wl, FP64, wl.steps, record_every=1,
                  per_step=lambda c, k: amps_g.append(np.fft.rfft(c.get_fields()[0][0].mean(axis=(0, 1)))[1]))
    amps_o = []
    F, osp, hist_o = run_oracle(wl, FP64, wl.steps,
                                per_step=lambda F, sp, k: amps_o.append(np.fft.rfft(F[0].mean(axis=(0, 1)))[1]))
    a_g, a_o = np.array(amps_g), np.array(amps_o)
    assert np.abs(a_g - a_o).max() <= 1e-9 * np.abs(a_o).max()
    t = np.arange(wl.steps) * wl.dt
    y = a_g.imag if np.abs(a_g.imag).max() > np.abs(a_g.real).max() else a_g.real
    y_o = a_o.imag if np.abs(a_o.imag).max() > np.abs(a_o.real).max() else a_o.real
    w_g, w_o = _fit(t, y), _fit(t, y_o)
    assert abs(w_g / w_o - 1) < 5e-3
    assert abs(w_g / w_o - 1) < 1e-6
    assert abs(w_g / oracle.cold_plasma_omega(2 * np.pi / 16, wl.dt) - 1) < 1e-5
    hist_g = ctx.history()
    assert hist_g.shape == hist_o.shape
    assert np.abs(hist_g.sum(1) / hist_o.sum(1) - 1).max() < 1e-9


@pytest.mark.parametrize("ppc,u_th", [(16, 0.05), (32, 0.1)])
def test_thermal_fp32_energy_history_within_one_percent(ppc, u_th):
    """FP32 bulk against the FP64 oracle over 100 steps of a 32^3 thermal plasma, in the
    shape of the 128^3 thermal workload (u_th = 0.05) and of the 256^3 precision-stress
    workload (32 per cell, u_th = 0.1): trajectories separate, the energy history agrees
    within 1%."""
    wl = W.thermal((32, 32, 32), 0.2, ppc, u_th, seed=10, steps=100)
    ctx = run_gpu(wl, FP32, wl.steps, track_ids=False, record_every=1)
    _, _, hist_o = run_oracle(wl, FP32, wl.steps)
    hist_g = ctx.history()
    tot_g, tot_o = hist_g.sum(1), hist_o.sum(1)
    assert np.abs(tot_g / tot_o - 1).max() < 1e-2
    assert np.abs(hist_g[:, 2] / hist_o[:, 2] - 1).max() < 1e-2


def test_cold_plasma_fp32_frequency():
    """The cold-plasma workload on the FP32 path (FP32-representable inputs on both
    sides): the frequency fitted to the Ex mode over 200 steps is within 0.5% of the
    oracle's (and of the closed-form discrete frequency)."""
    wl = _cold_plasma()
    wl.E = wl.E.astype(np.float32).astype(np.float64)
    amps_g = []
    run_gpu(wl, FP32, wl.steps,
            per_step=lambda c, k: amps_g.append(np.fft.rfft(c.get_fields()[0][0].mean(axis=(0, 1)))[1]))
    amps_o = []
    run_oracle(wl, FP32, wl.steps, per_step=lambda F, sp, k: amps_o.append(np.fft.rfft(F[0].mean(axis=(0, 1)))[1]))
    t = np.arange(wl.steps) * wl.dt
    a_g, a_o = np.array(amps_g), np.array(amps_o)
    pick = (lambda a: a.imag) if np.abs(a_o.imag).max() > np.abs(a_o.real).max() else (lambda a: a.real)
    w_g, w_o = _fit(t, pick(a_g)), _fit(t, pick(a_o))
    assert abs(w_g / w_o - 1) < 5e-3, (w_g, w_o)
    assert abs(w_g / oracle.cold_plasma_omega(2 * np.pi / 16, wl.dt) - 1) < 5e-3


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_continuity_and_gauss_on_device(prec):
    """Discrete continuity (Eq. (12)) and Gauss's law preservation measured by the
    library's FP64 reductions: continuity <= 1e-6 max|J| (FP32; ~1e-13 in FP64), Gauss
    change <= 1e-5 of max|rho| (FP32) over 30 steps."""
    wl = W.thermal((24, 24, 16), 0.2, 16, 0.1, seed=11)
    from paper_2609_16575_gb300 import gbpic

    sp = [W.SpeciesInput(s.q, s.m, W.quantize_fp32(s.P) if prec == FP32 else s.P) for s in wl.species]
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=False)
    ctx.set_fields(None, None)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P)
    d0 = ctx.diagnostics()
    assert np.isnan(d0["cont_max"])
    worst_cont = 0.0
    for k in range(30):
        ctx.step(1)
        dk = ctx.diagnostics()
        ratio = dk["cont_max"] * min(wl.d) / dk["J_max"]
        worst_cont = max(worst_cont, ratio)
    assert worst_cont <= (1e-6 if prec == FP32 else 1e-12), worst_cont
    assert dk["gauss_change_max"] <= (1e-5 if prec == FP32 else 1e-11) * dk["rho_max"]
    assert dk["n_alive"] == wl.nparticles


def test_diagnostics_match_oracle_sums():
    """pic_diagnostics' FP64 energies equal the oracle's sums on the same state."""
    wl = W.thermal((16, 16, 16), 0.2, 8, 0.2, seed=12)
    from pic_runs import plane_wave_fields

    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx = run_gpu(wl, FP64, 3)
    F, osp, _ = run_oracle(wl, FP64, 3)
    d = ctx.diagnostics()
    dv = np.prod(wl.d)
    Bn = F[3:6].copy()
    oracle.faraday(wl.n, wl.d, wl.dt, np.ascontiguousarray(F[0:3]), Bn, 0.5)
    assert abs(d["U_E"] / (0.5 * dv * (F[0:3] ** 2).sum()) - 1) < 1e-12
    assert abs(d["U_B"] / (0.5 * dv * (Bn ** 2).sum()) - 1) < 1e-12
    P = osp[0].P
    u2 = (P[3:6] ** 2).sum(0)
    K = (P[6] * u2 / (np.sqrt(1 + u2) + 1)).sum()
    assert abs(d["K_half"] / K - 1) < 1e-12
    rho = oracle.rho(wl.n, wl.d, osp, wl.rho_ion)
    G = oracle.divergence(wl.n, wl.d, F[0:3]) - rho
    assert abs(d["gauss_max"] / np.abs(G).max() - 1) < 1e-10


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_div_b_stays_zero(prec):
    """Faraday's law keeps div B at its initial value (zero here) on the GPU: a hot plasma
    under a divergence-free plane-wave B, 40 cycles."""
    from pic_runs import plane_wave_fields

    wl = W.thermal((16, 16, 8), 0.2, 4, 0.3, seed=141)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx = run_gpu(wl, prec, 40)
    E, B, _ = ctx.get_fields()
    div = oracle.divergence_b(wl.n, wl.d, B)
    scale = np.abs(B).max() / min(wl.d)
    assert np.abs(div).max() <= (1e-5 if prec == FP32 else 1e-13) * scale, np.abs(div).max() / scale
    assert np.abs(B).max() > 1e-3
    ctx.close()


def test_wakefield_plausible():
    """Plausibility of the laser wakefield (section 4: the peak accelerating field is
    about the cold wave-breaking field E_wb = omega_p m c / e): a short a0 = 2 pulse into
    n = 0.01 n_c with a moving window; the largest longitudinal field behind the pulse
    on the axis is of order E_wb = 0.1 (laser units)."""
    wl = W.lwfa(n=(256, 64, 64), ppc_per_dim=1, density=0.01, x0=20, ramp=20, a0=2.0, w0_lambda=2.0,
                fwhm_periods=4.0, plane=2, window_start=700)
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=FP32, rho_ion=0.0, bc_x=1)
    ctx.set_laser(*wl.laser.as_tuple())
    ctx.set_moving_window(*wl.window.as_tuple())
    s = wl.species[0]
    ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step)
    ctx.step(1400)
    E, _, _ = ctx.get_fields()
    ey = np.abs(E[1, 32, 32, :])
    front = int(np.argmax(ey))                          # the pulse
    ex = E[0, 32, 32, :max(front - 40, 1)]              # behind it
    e_wb = np.sqrt(0.01)
    assert ctx.window_moves() > 100
    assert 0.2 * e_wb < np.abs(ex).max() < 3.0 * e_wb, np.abs(ex).max() / e_wb
    ctx.close()
