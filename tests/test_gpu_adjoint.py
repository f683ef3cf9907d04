"""GPU adjoint (checkpointed, hand-written kernels) against an FP64 torch-autograd
reference of the same cycle and against central finite differences of the FP64 GPU
forward map.  Loss: final field energy; parameters: initial momenta u^{-1/2} and the
amplitude A of the initial plane-wave field."""
import numpy as np

import oracle
import pytest
import torch

from paper_2609_16575_gb300 import workloads as W
from pic_runs import plane_wave_fields
import torch_pic

pytestmark = pytest.mark.gpu


def _gpu_loss(wl, P, A, E_dir, B_dir, nsteps, ckpt, want_grad=True, sort_every=0, precision=None):
    from paper_2609_16575_gb300 import gbpic

    prec = gbpic.PIC_FP64 if precision is None else precision
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, track_ids=True, sort_every=sort_every)
    ctx.set_fields(A * E_dir, A * B_dir)
    ctx.load_species_array(-1.0, 1.0, P)
    L = ctx.adjoint_forward(nsteps, ckpt)
    out = (L,)
    if want_grad:
        dA, du = ctx.adjoint_backward(E_dir, B_dir)
        out = (L, dA, du[0])
    cells = np.floor(ctx.get_particles(0)[0:3])
    ctx.close()
    return out + (cells,)


@pytest.mark.parametrize("nsteps,ckpt,sort_every", [(20, 6, 0), (13, 13, 1), (9, 1, -1)])
def test_adjoint_matches_torch_autograd(nsteps, ckpt, sort_every):
    wl = W.thermal((4, 4, 4), 0.2, 2, 0.2, seed=31)
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    A = 0.05
    P = wl.species[0].P
    L, dA, du, _ = _gpu_loss(wl, P, A, E_dir, B_dir, nsteps, ckpt, sort_every=sort_every)
    Pt = torch.tensor(P).requires_grad_(True)
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    E, B, *_ = torch_pic.run(At * torch.tensor(E_dir), At * torch.tensor(B_dir), Pt, -1.0, 1.0, wl.n, wl.d, wl.dt,
                             nsteps)
    Lt = torch_pic.field_energy(E, B, wl.d, wl.dt)
    Lt.backward()
    Lv = float(Lt.detach())
    assert abs(L - Lv) <= 1e-12 * abs(Lv)
    g_ref = Pt.grad[3:6].numpy()
    assert np.abs(du - g_ref).max() <= 1e-8 * np.abs(g_ref).max()
    assert abs(dA - float(At.grad)) <= 1e-8 * abs(float(At.grad))


def test_adjoint_matches_central_differences():
    """Differentiable-run workload, reduced (16^3, 4 per cell, u_th = 0.02, plane wave,
    40 steps, checkpoints every 10): directional derivative along a random momentum
    direction and the amplitude derivative agree with central differences (perturbations
    small enough that no particle ends in another cell; the full-size test below checks
    the cells at every step)."""
    wl = W.differentiable(n=16, ppc=4, steps=40)
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    A = 0.05
    P = wl.species[0].P
    L, dA, du, cells = _gpu_loss(wl, P, A, E_dir, B_dir, 40, 10)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((3, P.shape[1]))
    h = 1e-7
    Pp, Pm = P.copy(), P.copy()
    Pp[3:6] += h * v
    Pm[3:6] -= h * v
    Lp, cp = _gpu_loss(wl, Pp, A, E_dir, B_dir, 40, 10, want_grad=False)
    Lm, cm = _gpu_loss(wl, Pm, A, E_dir, B_dir, 40, 10, want_grad=False)
    assert np.array_equal(cp, cm) and np.array_equal(cp, cells)
    fd = (Lp - Lm) / (2 * h)
    ad = float((du * v).sum())
    assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)
    hA = 1e-6 * A
    LAp, _ = _gpu_loss(wl, P, A + hA, E_dir, B_dir, 40, 10, want_grad=False)
    LAm, _ = _gpu_loss(wl, P, A - hA, E_dir, B_dir, 40, 10, want_grad=False)
    fdA = (LAp - LAm) / (2 * hA)
    assert abs(fdA - dA) <= 1e-4 * abs(dA), (fdA, dA)


def _cell_checksum(ctx, n, npart):
    """Two integer sums that change when any particle's half cell changes: sum of the
    linear half-cell index and sum of (id + 1) times it, from a device-side read-out
    (rows in id order).  Half cells, because the forward map has kinks there as well as
    at the faces: a half-located field component is interpolated from the samples on
    either side of the particle, which switch at offset 1/2."""
    import ctypes

    from paper_2609_16575_gb300 import gbpic

    out = torch.empty((7, npart), dtype=torch.float64, device="cuda")
    cnt = ctypes.c_int64(npart)
    assert gbpic.lib().pic_get_particles(ctx.ptr, 0, ctypes.c_void_p(out.data_ptr()), ctypes.byref(cnt), 1) == 0
    c = torch.floor(2.0 * out[0:3]).to(torch.int64)
    lin = (c[2] * (2 * n[1]) + c[1]) * (2 * n[0]) + c[0]
    ids = torch.arange(1, npart + 1, device="cuda", dtype=torch.int64)
    return int(lin.sum()), int((lin * ids).sum())


def _checked_forward(wl, P, A, E_dir, B_dir, nsteps):
    """The FP64 forward map: L = U_E + U_B after nsteps, and the per-step cell checksums."""
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP64, track_ids=True)
    ctx.set_fields(A * E_dir, A * B_dir)
    ctx.load_species_array(-1.0, 1.0, P)
    sums = []
    for _ in range(nsteps):
        ctx.step(1)
        sums.append(_cell_checksum(ctx, wl.n, P.shape[1]))
    d = ctx.diagnostics()
    ctx.close()
    return d["U_E"] + d["U_B"], sums


def test_adjoint_matches_central_differences_on_the_differentiable_run():
    """The differentiable-run workload at its full size: 32^3 cells, 16 per cell (524,288
    electrons), u_th = 0.02, plane wave of amplitude 0.05, 200 steps, checkpoints every 20.
    The adjoint's amplitude derivative and its momentum gradient along directions
    (on 2048 particles each) agree with central differences of the FP64 forward map to
    1e-4.  A perturbation
    counts only if no particle's half cell changes differently at any step (per-step
    checksums of the perturbed runs equal the unperturbed run's: the map has kinks at
    cell faces and at half cells); another direction, or a smaller step, is drawn
    otherwise."""
    wl = W.differentiable()
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    A = 0.05
    P = wl.species[0].P
    L, dA, du, _ = _gpu_loss(wl, P, A, E_dir, B_dir, 200, 20)
    L0, sums0 = _checked_forward(wl, P, A, E_dir, B_dir, 200)
    assert abs(L0 - L) <= 1e-12 * abs(L)
    # amplitude: the largest step of the list whose perturbed runs keep every cell
    for rel in (1e-8, 2e-9, 5e-10, 1e-10):
        hA = rel * A
        LAp, sp = _checked_forward(wl, P, A + hA, E_dir, B_dir, 200)
        LAm, sm = _checked_forward(wl, P, A - hA, E_dir, B_dir, 200)
        if sp == sums0 and sm == sums0:
            break
    else:
        pytest.fail("every amplitude step changed a cell crossing")
    fdA = (LAp - LAm) / (2 * hA)
    assert abs(fdA - dA) <= 1e-4 * abs(dA), (rel, fdA, dA)
    # momenta, along directions on 2048 random particles (a direction over every
    # particle shifts some crossing by a step almost surely at any usable h), with
    # random magnitudes and the signs of the adjoint's own components: the directional
    # derivative is then a sum of same-sign terms, large against the central
    # difference's noise (the FP64 forward map sums J with atomics in any order and
    # reproduces L only to about 1e-15; over 2h = 2e-8 that is ~1e-7, as large as 1e-4
    # of a random-sign sum), and a wrong sign or size of any component still shows
    rng = np.random.default_rng(6)
    checked = 0
    for attempt in range(8):
        v = np.zeros((3, P.shape[1]))
        pick = rng.choice(P.shape[1], 2048, replace=False)
        v[:, pick] = np.sign(du[:, pick]) * (0.5 + rng.random((3, pick.size)))
        h = (1e-8, 1e-8, 3e-9, 3e-9, 1e-9, 1e-9, 1e-9, 1e-9)[attempt]
        Pp, Pm = P.copy(), P.copy()
        Pp[3:6] += h * v
        Pm[3:6] -= h * v
        Lp, sp = _checked_forward(wl, Pp, A, E_dir, B_dir, 200)
        Lm, sm = _checked_forward(wl, Pm, A, E_dir, B_dir, 200)
        if sp != sums0 or sm != sums0:
            continue   # a crossing moved by a step: not a differentiable neighbourhood
        fd = (Lp - Lm) / (2 * h)
        ad = float((du * v).sum())
        assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)
        checked += 1
        if checked == 2:
            break
    assert checked >= 1


def test_autograd_function():
    """torch.autograd through the library's adjoint (FieldEnergyRun)."""
    from paper_2609_16575_gb300 import autodiff

    wl = W.thermal((8, 8, 8), 0.2, 2, 0.05, seed=33)
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    P = wl.species[0].P
    setup = dict(n=wl.n, d=wl.d, dt=wl.dt, q=-1.0, m=1.0, X=P[0:3], w=P[6], E_dir=E_dir, B_dir=B_dir, nsteps=12,
                 ckpt_every=5)
    u = torch.tensor(P[3:6], requires_grad=True)
    A = torch.tensor(0.05, dtype=torch.float64, requires_grad=True)
    L = autodiff.field_energy(u, A, setup)
    gu, gA = torch.autograd.grad(L, [u, A])
    L2, dA, du, _ = _gpu_loss(wl, P, 0.05, E_dir, B_dir, 12, 5)
    assert abs(float(L.detach()) - L2) <= 1e-13 * abs(L2)
    assert np.abs(gu.numpy() - du).max() <= 1e-13 * np.abs(du).max()
    assert abs(float(gA) - dA) <= 1e-13 * abs(dA)


def test_fp32_adjoint_against_fp64():
    """The FP32 path's adjoint (working-precision Jacobian products and particle adjoint
    state, FP64 field accumulation) against the FP64 adjoint on the same FP32-representable inputs:
    loss, momentum gradient and amplitude gradient within 1e-3 (the FP32 forward
    trajectory itself departs from the FP64 one at the 1e-6 level over 40 steps)."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.differentiable(n=16, ppc=4, steps=40)
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    E_dir = E_dir.astype(np.float32).astype(np.float64)
    B_dir = B_dir.astype(np.float32).astype(np.float64)
    A = 0.0625   # exact in FP32, so that A E_dir is too
    P = W.quantize_fp32(wl.species[0].P)
    L64, dA64, du64, _ = _gpu_loss(wl, P, A, E_dir, B_dir, 40, 10, precision=gbpic.PIC_FP64)
    L32, dA32, du32, _ = _gpu_loss(wl, P, A, E_dir, B_dir, 40, 10, precision=gbpic.PIC_FP32)
    assert abs(L32 - L64) <= 1e-5 * abs(L64)
    assert abs(dA32 - dA64) <= 1e-3 * abs(dA64), (dA32, dA64)
    assert np.abs(du32 - du64).max() <= 1e-3 * np.abs(du64).max(), np.abs(du32 - du64).max() / np.abs(du64).max()


def test_adjoint_run_is_forward_then_backward():
    """pic_adjoint_run gives the loss and gradients of forward + backward."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((4, 4, 4), 0.2, 2, 0.2, seed=35)
    E_dir, B_dir = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=1.0)
    A = 0.05
    P = wl.species[0].P
    L, dA, du, _ = _gpu_loss(wl, P, A, E_dir, B_dir, 12, 5)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP64, track_ids=True)
    ctx.set_fields(A * E_dir, A * B_dir)
    ctx.load_species_array(-1.0, 1.0, P)
    L2, dA2, du2 = ctx.adjoint_run(12, 5, E_dir, B_dir)
    ctx.close()
    assert L2 == pytest.approx(L, rel=1e-14)
    assert dA2 == pytest.approx(dA, rel=1e-12)
    assert np.abs(du2[0] - du).max() <= 1e-12 * np.abs(du).max()


def test_background_enters_the_gauss_residual():
    """pic_set_background: rho_max and gauss_max become max |rho + rho_ion| of the
    oracle's CIC charge of the same particles (E = 0, so G = -(rho + rho_ion)), and the
    Gauss reference is taken again at the next pic_diagnostics."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((8, 8, 8), 0.2, 2, 0.1, seed=36)
    P = wl.species[0].P
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP64, rho_ion=0.0)
    ctx.load_species_array(-1.0, 1.0, P)
    sp = [oracle.Species(-1.0, 1.0, P.copy())]
    for rho_ion in (0.0, 1.0, 0.25):
        if rho_ion:
            ctx.set_background(rho_ion)
        ref = np.abs(oracle.rho(wl.n, wl.d, sp, rho_ion)).max()
        d1 = ctx.diagnostics()
        d2 = ctx.diagnostics()
        for dd in (d1, d2):
            assert dd["rho_max"] == pytest.approx(ref, rel=1e-12, abs=1e-12)
            assert dd["gauss_max"] == pytest.approx(ref, rel=1e-12, abs=1e-12)
        assert d1["gauss_change_max"] == 0.0          # the reference is taken again here
        assert d2["gauss_change_max"] <= 1e-12 * ref  # nothing stepped (charge sums in any order)
    with pytest.raises(gbpic.PicError):
        ctx.set_background(float("nan"))
    ctx.close()
