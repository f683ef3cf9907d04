"""GPU parity of Esirkepov's deposit (Esirkepov 2001; section 2.5 names it next to the
ZigZag the paper uses) against the FP64 oracle: the tile kernel's crossers, the spill
list and the open x, on FP32 and FP64."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, oracle_n, prepare, rel_err, wrapped_diff

pytestmark = pytest.mark.gpu
ESK = dict(esirkepov=1)


def _ctx(wl, prec, scheme, slack=0.0):
    from paper_2609_16575_gb300 import gbpic

    sp, E, B = prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True, bc_x=wl.bc_x)
    ctx.set_deposit(scheme)
    ctx.set_fields(E, B)
    for s in sp:
        ctx.load_species_array(s.q, s.m, s.P, s.momenta_at_half_step, capacity_slack=slack)
    F = oracle.empty_fields(oracle_n(wl))
    if E is not None:
        F[0:3] = E
    if B is not None:
        F[3:6] = B
    return ctx, F, [oracle.Species(s.q, s.m, s.P.copy()) for s in sp]


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_esirkepov_hot_plasma(prec):
    """A hot periodic plasma (u_th = 0.3: a fifth of the particles cross a face every
    step) for 12 cycles: fields, J and every particle follow the oracle's Esirkepov run,
    and the current differs from the ZigZag run of the same state."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((24, 16, 8), 0.2, 4, 0.3, seed=101)
    ctx, F, osp = _ctx(wl, prec, gbpic.PIC_DEPOSIT_ESIRKEPOV)
    ctx.step(12)
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 12, guide=ESK)
    tol = 2e-5 if prec == FP32 else 1e-11
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])
    assert rel_err(J, F[6:9]) <= tol, rel_err(J, F[6:9])
    P = ctx.get_particles(0)
    Q = osp[0].P
    assert np.abs(wrapped_diff(P[0:3], Q[0:3], wl.n)).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert rel_err(P[3:6], Q[3:6]) <= tol
    # exact continuity of the GPU's own current (FP64: to round-off)
    ctx.diagnostics()
    ctx.step(1)
    d = ctx.diagnostics()
    assert d["cont_max"] * min(wl.d) <= (1e-6 if prec == FP32 else 1e-12) * d["J_max"]
    ctx.close()
    z, Fz, oz = _ctx(wl, prec, gbpic.PIC_DEPOSIT_ZIGZAG)
    z.step(12)
    _, _, Jz = z.get_fields()
    assert rel_err(Jz, J) > 1e-4
    z.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_esirkepov_relativistic_crossers(prec):
    """A relativistic plasma (u_th = 1, 16 per cell: about 30 % of the particles cross a
    face every step) for 4 cycles: the tile kernel's warps export every crosser's record
    in batches and k_esk_crossers deposits them once per step, against the oracle."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 16, 8), 0.2, 16, 1.0, seed=103)
    ctx, F, osp = _ctx(wl, prec, gbpic.PIC_DEPOSIT_ESIRKEPOV)
    ctx.set_timing(True)
    ctx.step(4)
    kt = ctx.kernel_times()
    assert kt["esk_crossers"][0] == 4
    oracle.run(wl.n, wl.d, wl.dt, F, osp, 4, guide=ESK)
    tol = 2e-5 if prec == FP32 else 1e-11
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])
    assert rel_err(J, F[6:9]) <= tol, rel_err(J, F[6:9])
    P = ctx.get_particles(0)
    assert np.abs(wrapped_diff(P[0:3], osp[0].P[0:3], wl.n)).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert rel_err(P[3:6], osp[0].P[3:6]) <= tol
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_esirkepov_spill_and_open_x(prec):
    """A fast beam into tiles that held nothing at load (the overflow is pushed from the
    spill list) leaving through the open face x = n: Esirkepov everywhere."""
    from paper_2609_16575_gb300 import gbpic

    n, d = (16, 8, 8), (0.2, 0.2, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    rng = np.random.Generator(np.random.PCG64(102))
    npart = 3000
    P = np.empty((7, npart))
    P[0] = rng.random(npart) * 6.0
    P[1] = rng.random(npart) * n[1]
    P[2] = rng.random(npart) * n[2]
    P[3] = 3.0 + 0.1 * rng.standard_normal(npart)
    P[4] = 0.3 * rng.standard_normal(npart)
    P[5] = 0.3 * rng.standard_normal(npart)
    P[6] = 1e-4
    wl = W.Workload("beam", n, d, dt, 0.0, [W.SpeciesInput(-1.0, 1.0, P)], bc_x=1)
    ctx, F, osp = _ctx(wl, prec, gbpic.PIC_DEPOSIT_ESIRKEPOV)
    ctx.step(45)
    oracle.run(oracle_n(wl), wl.d, wl.dt, F, osp, 45, guide=ESK)
    Pg = ctx.get_particles(0)
    Q = osp[0].P
    gone = Q[6] == 0.0
    assert npart // 4 < gone.sum() < npart * 3 // 4
    assert np.array_equal(np.isnan(Pg[6]), gone)
    keep = ~gone
    tol = 1e-4 if prec == FP32 else 1e-10
    assert np.abs(Pg[0:3, keep] - Q[0:3, keep]).max() <= tol
    assert rel_err(Pg[3:6, keep], Q[3:6, keep]) <= tol
    E, B, J = ctx.get_fields()
    assert rel_err(E, F[0:3]) <= tol, rel_err(E, F[0:3])
    assert rel_err(B, F[3:6]) <= tol, rel_err(B, F[3:6])
    ctx.close()


def test_deposit_argument_checks():
    from paper_2609_16575_gb300 import gbpic

    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, track_ids=True)
    with pytest.raises(gbpic.PicError):
        c.set_deposit(2)
    c.set_deposit(gbpic.PIC_DEPOSIT_ESIRKEPOV)
    c.load_species_array(-1.0, 1.0, np.array([[1.5], [1.5], [1.5], [0.1], [0.0], [0.0], [1e-3]]), True)
    with pytest.raises(gbpic.PicError):
        c.adjoint_forward(4, 2)            # the adjoint differentiates ZigZag only
    c.set_deposit(gbpic.PIC_DEPOSIT_ZIGZAG)
    c.step(1)
    c.sync()
    c.close()
