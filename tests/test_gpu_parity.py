"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances (normwise max relative error per array): <= 1e-5 for the
FP32 path and <= 1e-12 for the FP64 path after one step."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, plane_wave_fields, rel_err, run_gpu, run_oracle, wrapped_diff

pytestmark = pytest.mark.gpu

TOL = {FP32: 1e-5, FP64: 1e-12}


def _thermal(n, ppc=8, u_th=0.1, seed=3, d=0.2, fields=True):
    wl = W.thermal(n, d, ppc, u_th, seed=seed)
    if fields:
        wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    return wl


def _compare_state(ctx, F, osp, wl, prec, tol_f, tol_x, tol_u, joint_em=False):
    """joint_em: normalise E and B errors by the larger of max|E|, max|B| (for problems
    where one of them is only rounding noise)."""
    E, B, J = ctx.get_fields()
    if joint_em:
        scale = max(np.abs(F[0:3]).max(), np.abs(F[3:6]).max())
        assert np.abs(E - F[0:3]).max() <= tol_f * scale
        assert np.abs(B - F[3:6]).max() <= tol_f * scale
    else:
        assert rel_err(E, F[0:3]) <= tol_f, ("E", rel_err(E, F[0:3]))
        assert rel_err(B, F[3:6]) <= tol_f, ("B", rel_err(B, F[3:6]))
    assert rel_err(J, F[6:9]) <= tol_f, ("J", rel_err(J, F[6:9]))
    for s, o in enumerate(osp):
        P = ctx.get_particles(s)
        assert P.shape == o.P.shape
        dx = np.abs(wrapped_diff(P[0:3], o.P[0:3], wl.n)).max()
        assert dx <= tol_x, ("X", dx)
        assert rel_err(P[3:6], o.P[3:6]) <= tol_u, ("u", rel_err(P[3:6], o.P[3:6]))
        assert np.array_equal(P[6], o.P[6])


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("n", [(16, 16, 16), (20, 16, 12), (9, 17, 5)])
def test_one_step_thermal(prec, n):
    """One cycle on a thermal plasma with a plane-wave field: several tiles, ragged
    edge tiles, particles crossing cells and the periodic boundary."""
    wl = _thermal(n)
    ctx = run_gpu(wl, prec, 1)
    F, osp, _ = run_oracle(wl, prec, 1)
    tol = TOL[prec]
    _compare_state(ctx, F, osp, wl, prec, tol, 1e-6 if prec == FP32 else 1e-13, tol, )


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_ten_steps_thermal(prec):
    wl = _thermal((16, 24, 16), ppc=4, u_th=0.2, seed=4)
    ctx = run_gpu(wl, prec, 10)
    F, osp, _ = run_oracle(wl, prec, 10)
    tol = 2e-4 if prec == FP32 else 1e-10
    _compare_state(ctx, F, osp, wl, prec, tol, 1e-4 if prec == FP32 else 1e-11, tol)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_vacuum_plane_waves(prec):
    """No particles: the Yee kernels advance discrete eigenmodes like the closed form."""
    n, d = (24, 16, 8), (0.3, 0.25, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    E0, B0 = plane_wave_fields(n, d, dt, amplitude=0.3,
                               modes=(((1, 0, 0), (0, 1, 0)), ((0, 1, 1), None), ((2, -1, 1), None)))
    wl = W.Workload("vacuum", n, d, dt, 0.0, [], E0, B0)
    ctx = run_gpu(wl, prec, 40)
    F, _, _ = run_oracle(wl, prec, 40)
    E, B, J = ctx.get_fields()
    tol = 1e-5 if prec == FP32 else 1e-12
    assert rel_err(E, F[0:3]) <= tol
    assert rel_err(B, F[3:6]) <= tol
    assert np.abs(J).max() == 0.0


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_backpush_from_t0(prec):
    """Momenta given at t = 0: the library's backward half push matches the oracle's."""
    wl = _thermal((16, 16, 8), ppc=4, u_th=0.3, seed=5)
    for s in wl.species:
        s.momenta_at_half_step = False
    ctx = run_gpu(wl, prec, 1)
    F, osp, _ = run_oracle(wl, prec, 1)
    _compare_state(ctx, F, osp, wl, prec, TOL[prec], 1e-6 if prec == FP32 else 1e-13, TOL[prec])


def test_paper_grid_smaller_than_a_tile():
    """The paper's 2 x 2 x 100 plasma-oscillation grid: two dimensions smaller than a
    tile and a ragged last tile; 20 FP64 cycles."""
    wl = W.paper_cold_plasma(steps=20)
    ctx = run_gpu(wl, FP64, 20)
    F, osp, _ = run_oracle(wl, FP64, 20)
    _compare_state(ctx, F, osp, wl, FP64, 1e-11, 1e-12, 1e-11, joint_em=True)


def test_boundary_offsets_and_corners():
    """Particles exactly on cell faces (offset 0), at the top of a cell, and crossing
    the periodic corner of the box in all three dimensions."""
    n, d = (8, 16, 8), (0.2, 0.2, 0.2)
    dt = oracle.courant_dt(d, 0.5)
    X = np.array([[0.0, 7.999999, 3.0, 0.5, 7.9, 4.0],
                  [0.0, 15.999999, 8.0, 0.5, 15.95, 8.0],
                  [0.0, 7.999999, 4.0, 0.5, 7.9, 0.0]])
    u = np.array([[-0.9, 0.9, 0.5, 0.0, 2.0, -0.3],
                  [-0.9, 0.9, -0.5, 0.0, 2.0, 0.0],
                  [-0.9, 0.9, 0.2, 0.0, 2.0, -0.7]])
    P = np.vstack([X, u, np.full((1, 6), 1e-3)])
    wl = W.Workload("corners", n, d, dt, 0.0, [W.SpeciesInput(-1.0, 1.0, P)])
    wl.E, wl.B = plane_wave_fields(n, d, dt)
    for prec in (FP32, FP64):
        ctx = run_gpu(wl, prec, 3)
        F, osp, _ = run_oracle(wl, prec, 3)
        _compare_state(ctx, F, osp, wl, prec, 1e-5 if prec == FP32 else 1e-12, 1e-5 if prec == FP32 else 1e-12,
                       1e-5 if prec == FP32 else 1e-12)


def test_empty_species_and_two_species():
    """An empty species is legal; two species with different q/m push independently
    and their currents add."""
    wl = _thermal((16, 8, 8), ppc=4, seed=6)
    ions = W.thermal((16, 8, 8), 0.2, 2, 0.01, seed=7).species[0]
    ions.q, ions.m = 1.0, 100.0
    empty = W.SpeciesInput(-1.0, 1.0, np.zeros((7, 0)))
    wl.species = [wl.species[0], empty, ions]
    for prec in (FP32, FP64):
        ctx = run_gpu(wl, prec, 2)
        F, osp, _ = run_oracle(wl, prec, 2)
        tol = 1e-5 if prec == FP32 else 1e-12
        E, B, J = ctx.get_fields()
        assert rel_err(J, F[6:9]) <= tol
        assert rel_err(E, F[0:3]) <= tol
        assert ctx.get_particles(1).shape == (7, 0)
        P = ctx.get_particles(2)
        assert rel_err(P[3:6], osp[2].P[3:6]) <= tol


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_spill_path_matches(prec):
    """Converging flow with almost no segment headroom: tiles overflow, particles go
    through the spill list, and the result still matches the oracle."""
    n = (32, 8, 8)
    wl = W.thermal(n, 0.2, 8, 0.01, seed=8)
    P = wl.species[0].P
    P[3] = -0.6 * np.sign(P[0] - n[0] / 2)           # everyone streams towards x = L/2
    ctx = run_gpu(wl, prec, 12, slack=1e-6)
    diag = ctx.diagnostics()
    assert diag["n_spilled"] > 0                      # the spill path was exercised
    assert diag["n_alive"] == P.shape[1]
    F, osp, _ = run_oracle(wl, prec, 12)
    tol = 1e-4 if prec == FP32 else 1e-11
    _compare_state(ctx, F, osp, wl, prec, tol, 1e-4 if prec == FP32 else 1e-11, tol)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_segments_stay_grouped_by_cell(prec):
    """Every step writes each tile's particles grouped by the cell they started the step
    in, so after several steps with many cell crossings the segments read in slot order
    are grouped by cell except for the last step's crossers and the appended movers (the
    parity of the state itself is checked by the other tests)."""
    from paper_2609_16575_gb300 import gbpic

    wl = _thermal((16, 16, 16), ppc=16, u_th=0.2, seed=9)
    sp, E, B = __import__("pic_runs").prepare(wl, prec)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=False)
    ctx.set_fields(E, B)
    ctx.load_species_array(sp[0].q, sp[0].m, sp[0].P)
    ctx.step(7)
    assert ctx.diagnostics()["n_alive"] == sp[0].P.shape[1]
    Q = ctx.get_particles(0)                       # tile order, slots in order
    c = np.floor(Q[0:3]).astype(np.int64)
    tile = (c[2] // 8 * 2 + c[1] // 8) * 2 + c[0] // 8
    local = (c[0] % 8) | ((c[1] % 8) << 3) | ((c[2] % 8) << 6)
    assert np.all(np.diff(tile) >= 0)             # tile segments in tile order
    same = np.diff(tile) == 0
    descents = np.count_nonzero(np.diff(local)[same] < 0)
    # a random order would descend about half the time; u_th = 0.2 moves ~15 % of the
    # particles to another cell per step
    assert descents <= 0.2 * Q.shape[1], (descents, Q.shape[1])


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("deposit", [0, 1])
def test_graph_replayed_cycles_match_direct_steps(prec, deposit):
    """pic_step runs the middle cycles of a long call as a replayed two-cycle CUDA graph
    (periodic box, no history or timing): 13 cycles in one call against 13 calls of one
    cycle (no graph), on a grid of fewer tiles than SMs (split tiles) with a fifth of the
    particles crossing a face per step.  The runs agree to the path's rounding (the order
    of a cell's particles in its range, hence the grouping of their FP32 partial sums or
    of the FP64 atomic additions, varies from run to run): 1e-5 / 1e-12 of each array's
    maximum.  The launch count and the step count advance as for direct steps."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((24, 16, 16), 0.2, 8, 0.3, seed=41)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt)
    out = []
    for calls in ((13,), (1,) * 13):
        ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True)
        ctx.set_deposit(deposit)
        ctx.set_fields(wl.E, wl.B)
        ctx.load_species_array(-1.0, 1.0, wl.species[0].P, False)
        l0 = ctx.launch_count()
        for k in calls:
            ctx.step(k)
        d = ctx.diagnostics()
        out.append((ctx.get_fields(), ctx.get_particles(0), ctx.launch_count() - l0, d["step"]))
        ctx.close()
    (Fa, Pa, La, Sa), (Fb, Pb, Lb, Sb) = out
    assert Sa == Sb == 13 and La == Lb
    tol = 1e-5 if prec == FP32 else 1e-12
    for a, b in zip(Fa, Fb):
        assert rel_err(a, b) <= tol
    assert np.abs(wrapped_diff(Pa[0:3], Pb[0:3], wl.n)).max() <= tol * max(wl.n)
    assert rel_err(Pa[3:6], Pb[3:6]) <= tol
