"""GPU adjoint (checkpointed, hand-written kernels) against an FP64 torch-autograd
reference of the same cycle and against central finite differences of the FP64 GPU
forward map.  Loss: final field energy; parameters: initial momenta u^{-1/2} and the
amplitude A of the initial plane-wave field."""
import numpy as np
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
    small enough that no particle's cell-crossing pattern changes; checked)."""
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
    """The FP32 path's adjoint (working-precision Jacobian products, FP64 adjoint state
    and accumulation) against the FP64 adjoint on the same FP32-representable inputs:
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
    """pic_set_background changes rho_max by the background, as a uniform charge does."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((8, 8, 8), 0.2, 2, 0.1, seed=36)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=gbpic.PIC_FP64, rho_ion=0.0)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    r0 = ctx.diagnostics()["rho_max"]
    ctx.set_background(1.0)
    d1 = ctx.diagnostics()
    assert d1["rho_max"] < r0            # the ions neutralise the electrons' charge
    with pytest.raises(gbpic.PicError):
        ctx.set_background(float("nan"))
    ctx.close()
