"""The allocation-free Gauss check (pic_gauss_check_static), for callers that cannot
allocate device memory (their pool owns it, or they must not trigger the
synchronisation of cudaMalloc/cudaFree).  Called twice in a row through the C ABI,
it must match pic_diagnostics' gauss_max and rho_max, allocate nothing, and refuse
grids beyond its static maximum.  Kept in a file of its own that pytest collects
last."""
import ctypes

import numpy as np
import pytest

from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, plane_wave_fields

pytestmark = pytest.mark.gpu

TOL = 1e-12   # both are FP64 reductions of the same quantities; only atomic order differs


@pytest.mark.parametrize("prec,bc_x", [(FP32, 0), (FP64, 0), (FP32, 1), (FP64, 1)])
def test_static_gauss_check_matches_diagnostics(prec, bc_x):
    """Periodic box, and an open x (bc_x = 1: the face node x = n has no charge slot and
    particles leave through both faces) where the charge scatter drops that node."""
    import torch
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((24, 16, 16), 0.2, 8, 0.2, seed=41)
    E, B = plane_wave_fields(wl.n, wl.d, wl.dt)
    if bc_x:   # an open x line holds n + 1 nodes of Ey, Ez, Bx: no field on the face
        E = np.concatenate([E, np.zeros(E.shape[:-1] + (1,))], axis=-1)
        B = np.concatenate([B, np.zeros(B.shape[:-1] + (1,))], axis=-1)
    P = W.quantize_fp32(wl.species[0].P) if prec == FP32 else wl.species[0].P
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, bc_x=bc_x)
    ctx.set_fields(E, B)
    ctx.load_species_array(-1.0, 1.0, P)
    ctx.step(3)
    ctx.sync()
    torch.cuda.synchronize()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    L = gbpic.lib()
    results = []
    for _ in range(2):          # two calls in a row share the static scratch
        g, r = ctypes.c_double(), ctypes.c_double()
        assert L.pic_gauss_check_static(ctx.ptr, ctypes.byref(g), ctypes.byref(r)) == 0
        results.append((g.value, r.value))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
    ref = ctx.diagnostics()       # the existing entry point (allocates its own scratch)
    for g, r in results:
        assert abs(g - ref["gauss_max"]) <= TOL * ref["gauss_max"]
        assert abs(r - ref["rho_max"]) <= TOL * ref["rho_max"]
    ctx.close()


def test_static_gauss_check_rejects_large_grids():
    from paper_2609_16575_gb300 import gbpic

    ctx = gbpic.Context((128, 128, 128), (0.2, 0.2, 0.2), 0.05, precision=FP32)
    g, r = ctypes.c_double(), ctypes.c_double()
    status = gbpic.lib().pic_gauss_check_static(ctx.ptr, ctypes.byref(g), ctypes.byref(r))
    assert status == 1                                   # PIC_ERR_ARG
    assert b"maximum" in gbpic.lib().pic_last_error(ctx.ptr)
    ctx.close()
