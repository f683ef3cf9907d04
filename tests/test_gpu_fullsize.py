"""Full-size parity on the thermal-plasma workload (128^3 cells, 64 electrons per cell,
~134M particles, FP32) in the launch configuration the benchmark times (no particle
ids).  The oracle recomputes two 8^3-cell sub-regions exactly (every particle whose
zigzag footprint can reach them is included); continuity and particle conservation
are checked on the whole grid by the library's FP64 reductions."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from pic_runs import FP32, FP64, plane_wave_fields

pytestmark = pytest.mark.gpu


def _region_check(wl, P32, E0, B0, Eg, Bg, Jg, lo, tol=1e-5):
    """Oracle step on the particles within 2 cells of the 8^3 region starting at lo
    (periodic); compare J and E there and B everywhere."""
    n = wl.n
    c = np.floor(P32[0:3]).astype(np.int64)
    sel = np.ones(P32.shape[1], dtype=bool)
    for k in range(3):
        rel = (c[k] - (lo[k] - 2)) % n[k]
        sel &= rel < 12
    sub = oracle.Species(-1.0, 1.0, np.ascontiguousarray(P32[:, sel]))
    F = oracle.empty_fields(n)
    F[0:3] = E0
    F[3:6] = B0
    oracle.run(n, wl.d, wl.dt, F, [sub], 1)
    idx = np.ix_(*(((np.arange(8) + lo[k]) % n[k]) for k in (2, 1, 0)))
    for comp in range(3):
        ref = F[6 + comp][idx]
        got = Jg[comp][idx]
        assert np.abs(got - ref).max() <= tol * np.abs(Jg[comp]).max()
        refE = F[comp][idx]
        assert np.abs(Eg[comp][idx] - refE).max() <= tol * np.abs(Eg[comp]).max()
    assert np.abs(Bg - F[3:6]).max() <= tol * np.abs(F[3:6]).max()
    return sel.sum()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_thermal128_one_step(prec):
    """One cycle of the full 128^3 x 64 workload; FP32 within 1e-5, the FP64 path within
    1e-12 of the oracle on two sub-regions."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal()
    E0, B0 = plane_wave_fields(wl.n, wl.d, wl.dt)
    if prec == FP32:
        E0 = E0.astype(np.float32).astype(np.float64)
        B0 = B0.astype(np.float32).astype(np.float64)
    P = wl.species[0].P
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=False)
    ctx.set_fields(E0, B0)
    ctx.load_species_array(-1.0, 1.0, P)
    d0 = ctx.diagnostics()
    ctx.step(1)
    d1 = ctx.diagnostics()
    assert d1["n_alive"] == P.shape[1]
    assert d1["cont_max"] * min(wl.d) <= (1e-6 if prec == FP32 else 1e-12) * d1["J_max"]
    Eg, Bg, Jg = ctx.get_fields()
    ctx.close()
    Pin = W.quantize_fp32(P) if prec == FP32 else P
    del P, wl.species[0].P
    used = 0
    for lo in ((40, 64, 16), (124, 0, 121)):          # the second region wraps the box
        used += _region_check(wl, Pin, E0, B0, Eg, Bg, Jg, lo, tol=1e-5 if prec == FP32 else 1e-12)
    assert used > 100000
