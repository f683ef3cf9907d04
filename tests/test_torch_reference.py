"""Pins of the FP64 torch-autograd gradient reference (tests/torch_pic.py): its forward
map equals the oracle's, and its autograd gradient equals central finite differences."""
import numpy as np
import torch

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import plane_wave_fields
import torch_pic


def _case(seed=21):
    wl = W.thermal((4, 4, 4), 0.2, 2, 0.2, seed=seed)
    wl.E, wl.B = plane_wave_fields(wl.n, wl.d, wl.dt, amplitude=0.05)
    return wl


def test_torch_reference_forward_equals_oracle():
    wl = _case()
    P = wl.species[0].P
    E, B, C, x, u = torch_pic.run(torch.tensor(wl.E), torch.tensor(wl.B), torch.tensor(P), -1.0, 1.0, wl.n, wl.d,
                                  wl.dt, 6)
    F = oracle.empty_fields(wl.n)
    F[0:3], F[3:6] = wl.E, wl.B
    sp = [oracle.Species(-1.0, 1.0, P)]
    oracle.run(wl.n, wl.d, wl.dt, F, sp, 6)
    assert np.abs(E.numpy() - F[0:3]).max() < 1e-13
    assert np.abs(B.numpy() - F[3:6]).max() < 1e-13
    assert np.array_equal(C.numpy(), sp[0].C.astype(np.int64))
    assert np.abs(x.numpy() - sp[0].Q[0:3]).max() < 1e-13
    assert np.abs(u.numpy() - sp[0].Q[3:6]).max() < 1e-13


def test_torch_reference_gradient_is_finite_difference():
    wl = _case(seed=22)
    P0 = torch.tensor(wl.species[0].P)
    E0, B0 = torch.tensor(wl.E), torch.tensor(wl.B)

    def loss(Pt, A):
        E, B, *_ = torch_pic.run(A * E0, A * B0, Pt, -1.0, 1.0, wl.n, wl.d, wl.dt, 5)
        return torch_pic.field_energy(E, B, wl.d, wl.dt)

    P = P0.clone().requires_grad_(True)
    A = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    L = loss(P, A)
    L.backward()
    rng = np.random.default_rng(1)
    v = torch.zeros_like(P0)
    v[3:6] = torch.tensor(rng.standard_normal((3, P0.shape[1])))
    h = 1e-6
    with torch.no_grad():
        fd = (loss(P0 + h * v, A) - loss(P0 - h * v, A)) / (2 * h)
        fdA = (loss(P0, A + h) - loss(P0, A - h)) / (2 * h)
    ad = (P.grad * v).sum()
    assert abs(float(fd - ad)) <= 1e-6 * abs(float(ad))
    assert abs(float(fdA - A.grad)) <= 1e-6 * abs(float(A.grad))
