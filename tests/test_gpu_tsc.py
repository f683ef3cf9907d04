"""The quadratic (TSC) particle shape on the GPU against the FP64 oracle (section 2.5,
Eq. (16) with the first-order cloud b1; section 5): one cycle at the single-step parity
tolerances (every field array and the particle state within 1e-5 on the FP32 path,
1e-12 on the FP64 path) on grids of several tiles with ragged edges, tiny grids whose
support wraps onto itself, the back-push, the spill path, twenty cycles on the FP64
path, the diagnostics' TSC charge (Gauss's law and continuity), the benchmark-sized
128^3 x 64 thermal plasma on sampled sub-regions, and the API's restrictions."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, plane_wave_fields, prepare, rel_err, wrapped_diff

pytestmark = pytest.mark.gpu

TOL = {FP32: 1e-5, FP64: 1e-12}
TSC = {"shape": 2}


def _start(wl, prec, slack=0.0, backpush=False):
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True)
    ctx.set_shape(gbpic.PIC_SHAPE_TSC)
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, not backpush, capacity_slack=slack)
    F = oracle.empty_fields(wl.n)
    if E is not None:
        F[0:3] = E
    if B is not None:
        F[3:6] = B
    osp = [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]
    if backpush:
        for s in osp:
            oracle.backpush(wl.n, wl.d, wl.dt, F[0:3], F[3:6], s, shape=2)
    return ctx, F, osp


def _compare(ctx, F, osp, wl, tol):
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, ("E", rel_err(E, F[0:3]))
    assert rel_err(B, F[3:6]) <= tol, ("B", rel_err(B, F[3:6]))
    assert rel_err(J, F[6:9]) <= tol, ("J", rel_err(J, F[6:9]))
    P = ctx.get_particles(0)
    Q = osp[0].P
    assert P.shape == Q.shape
    assert np.abs(wrapped_diff(P[0:3], Q[0:3], wl.n)).max() <= tol * max(wl.n)
    assert rel_err(P[3:6], Q[3:6]) <= tol


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("n", [(24, 16, 8), (21, 13, 10), (3, 5, 2)])
def test_one_tsc_cycle(prec, n):
    """Several tiles with ragged edges, and a grid smaller than the shape's support
    (the 27 samples and the 4 x 4 x 4 deposit wrap onto themselves)."""
    wl = W.thermal(n, 0.2, 6, 0.3, seed=301)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx, F, osp = _start(wl, prec)
    ctx.step(1)
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 1, guide=TSC)
    _compare(ctx, F, osp, wl, TOL[prec])
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_tsc_backpush_and_spill_path(prec):
    """Momenta given at t = 0 (the TSC back-push) and a converging flow with almost no
    segment headroom: tiles overflow and particles go through the spill list."""
    n = (32, 8, 8)
    wl = W.thermal(n, 0.2, 8, 0.01, seed=302)
    P = wl.species[0].P
    P[3] = -0.6 * np.sign(P[0] - n[0] / 2)            # everyone streams towards x = L/2
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx, F, osp = _start(wl, prec, slack=1e-6, backpush=True)
    ctx.step(12)
    d = ctx.diagnostics()
    assert d["n_spilled"] > 0 and d["n_alive"] == P.shape[1]
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 12, guide=TSC)
    _compare(ctx, F, osp, wl, 1e-4 if prec == FP32 else 1e-11)
    ctx.close()


def test_tsc_twenty_cycles_fp64():
    wl = W.thermal((16, 16, 16), 0.2, 8, 0.1, seed=303)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    ctx, F, osp = _start(wl, FP64)
    ctx.step(20)
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 20, guide=TSC)
    _compare(ctx, F, osp, wl, 1e-11)
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_tsc_diagnostics_keep_gauss_and_continuity(prec):
    """The library's FP64 diagnostics take the TSC charge: the Gauss residual keeps its
    initial value and the continuity residual vanishes, as with CIC; the charge maximum
    equals the oracle's TSC charge of the same particles."""
    wl = W.thermal((24, 16, 16), 0.2, 8, 0.1, seed=304)
    ctx, F, osp = _start(wl, prec)
    d0 = ctx.diagnostics()
    rho_ref = oracle.rho(wl.n, wl.d, osp, rho_ion=wl.rho_ion, shape=2)
    assert d0["rho_max"] == pytest.approx(np.abs(rho_ref).max(), rel=1e-6 if prec == FP32 else 1e-12)
    for _ in range(5):
        ctx.step(1)
        d = ctx.diagnostics()
        bound = 1e-5 if prec == FP32 else 1e-12
        assert d["gauss_change_max"] <= bound * d["rho_max"]
        assert d["cont_max"] * min(wl.d) <= (1e-6 if prec == FP32 else 1e-12) * d["J_max"]
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_tsc_full_size_thermal128_regions(prec):
    """One cycle of the 128^3 x 64 thermal plasma with TSC: the oracle recomputes two
    8^3 sub-regions from every particle whose support can reach them (within 3 cells)."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal()
    E0, B0 = plane_wave_fields(wl.n, wl.d, wl.dt)
    if prec == FP32:
        E0 = E0.astype(np.float32).astype(np.float64)
        B0 = B0.astype(np.float32).astype(np.float64)
    P = wl.species[0].P
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=False)
    ctx.set_shape(gbpic.PIC_SHAPE_TSC)
    ctx.set_fields(E0, B0)
    ctx.load_species_array(-1.0, 1.0, P)
    ctx.step(1)
    d1 = ctx.diagnostics()
    assert d1["n_alive"] == P.shape[1]
    Eg, Bg, Jg = ctx.get_fields()
    ctx.close()
    Pin = W.quantize_fp32(P) if prec == FP32 else P
    del P, wl.species[0].P
    tol = TOL[prec]
    n = wl.n
    c = np.floor(Pin[0:3]).astype(np.int64)
    for lo in ((40, 64, 16), (124, 0, 121)):
        sel = np.ones(Pin.shape[1], dtype=bool)
        for k in range(3):
            sel &= ((c[k] - (lo[k] - 3)) % n[k]) < 14
        sub = oracle.Species(-1.0, 1.0, np.ascontiguousarray(Pin[:, sel]))
        F = oracle.empty_fields(n)
        F[0:3] = E0
        F[3:6] = B0
        oracle.run(n, wl.d, wl.dt, F, [sub], 1, guide=TSC)
        idx = np.ix_(*(((np.arange(8) + lo[k]) % n[k]) for k in (2, 1, 0)))
        for comp in range(3):
            assert np.abs(Jg[comp][idx] - F[6 + comp][idx]).max() <= tol * np.abs(Jg[comp]).max()
            assert np.abs(Eg[comp][idx] - F[comp][idx]).max() <= tol * np.abs(Eg[comp]).max()
        assert np.abs(Bg - F[3:6]).max() <= tol * np.abs(F[3:6]).max()


def test_tsc_restrictions():
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=1)
    with pytest.raises(gbpic.PicError) as e:
        ctx.set_shape(gbpic.PIC_SHAPE_TSC)
    assert e.value.status == gbpic.PIC_ERR_STATE
    ctx.close()
    wl = W.thermal((8, 8, 8), 0.2, 2, 0.05, seed=305)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, rho_ion=1.0, track_ids=True)
    with pytest.raises(gbpic.PicError) as e:
        ctx.set_shape(3)
    assert e.value.status == gbpic.PIC_ERR_ARG
    ctx.set_shape(gbpic.PIC_SHAPE_TSC)
    with pytest.raises(gbpic.PicError) as e:
        ctx.set_pec(1, 0)
    assert e.value.status == gbpic.PIC_ERR_STATE
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError) as e:
        ctx.adjoint_forward(4, 2)
    assert e.value.status == gbpic.PIC_ERR_STATE
    ctx.set_shape(gbpic.PIC_SHAPE_CIC)
    ctx.step(1)
    ctx.close()
