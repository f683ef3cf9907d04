"""Failure detection on the device without faulting it: bad inputs that the kernels
detect set an error bit, the next synchronising call returns the status, and the
process can carry on with a fresh context."""
import numpy as np
import pytest

from paper_2609_16575_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(gbpic, wl, prec):
    return gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True)


@pytest.mark.parametrize("prec", [0, 1])
def test_non_finite_momentum_is_reported(prec):
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=71)
    P = wl.species[0].P.copy()
    P[4, 17] = np.nan
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, P)
    with pytest.raises(gbpic.PicError) as e:
        ctx.step(2)
        ctx.sync()
    assert e.value.status == gbpic.PIC_ERR_NAN
    ctx.close()
    # a fresh context on the same device works
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    ctx.step(2)
    ctx.sync()
    assert ctx.diagnostics()["n_alive"] == wl.species[0].P.shape[1]
    ctx.close()


def test_positions_outside_the_box_are_rejected_at_load():
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=72)
    P = wl.species[0].P.copy()
    P[1, 3] = 8.0          # y = n_y is outside [0, n_y)
    ctx = _ctx(gbpic, wl, 0)
    with pytest.raises(gbpic.PicError) as e:
        ctx.load_species_array(-1.0, 1.0, P)
    assert e.value.status == gbpic.PIC_ERR_ARG
    P[1, 3] = 7.5
    P[6, 5] = -1.0         # weights must be positive
    with pytest.raises(gbpic.PicError) as e:
        ctx.load_species_array(-1.0, 1.0, P)
    assert e.value.status == gbpic.PIC_ERR_ARG
    ctx.close()


def test_adjoint_needs_ids_and_a_periodic_box():
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=73)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=1, rho_ion=wl.rho_ion, track_ids=False)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError):
        ctx.adjoint_forward(4, 2)
    ctx.close()
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=1, rho_ion=0.0, track_ids=True, bc_x=1)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError):
        ctx.adjoint_forward(4, 2)
    ctx.close()
