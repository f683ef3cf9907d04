"""GPU parity of the perfectly conducting wall planes and the waveguide port (section 3.2:
the Yee solver is verified on the TE10 mode of a conducting rectangular guide driven at
its input plane) against the FP64 oracle and the exact discrete mode."""
import numpy as np
import pytest

import oracle
from pic_runs import FP32, FP64, rel_err
from test_oracle_guide import _te_mode

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_te10_mode_of_the_guide(prec):
    """The exact discrete TE10 mode of a guide closed by the wall planes y = 0 and z = 0
    (periodic x): after 300 steps the library matches the closed form and the oracle."""
    from paper_2609_16575_gb300 import gbpic

    n, d = (16, 12, 4), (0.1, 0.13, 0.1)
    dt = oracle.courant_dt(d, 0.5)
    E, B, w, kx, ky = _te_mode(n, d, dt, 2, 1)
    if prec == FP32:
        E, B = E.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    steps = 300
    ctx = gbpic.Context(n, d, dt, precision=prec)
    ctx.set_pec(1, 1)
    ctx.set_fields(E, B)
    ctx.step(steps)
    Eg, Bg, _ = ctx.get_fields()
    F = oracle.empty_fields(n)
    F[0:3], F[3:6] = E, B
    oracle.run(n, d, dt, F, [], steps, guide=dict(pec_y=1, pec_z=1))
    tol = 2e-5 if prec == FP32 else 1e-12
    assert rel_err(Eg, F[0:3]) <= tol, rel_err(Eg, F[0:3])
    assert rel_err(Bg, F[3:6]) <= tol, rel_err(Bg, F[3:6])
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    ref = np.sin(ky * jj * d[1]) * np.sin(kx * ii * d[0] - w * steps * dt)
    assert np.abs(Eg[2] - ref).max() <= (1e-4 if prec == FP32 else 1e-11)
    assert np.abs(Eg[2][:, 0, :]).max() == 0.0 and np.abs(Eg[0]).max() == 0.0
    ctx.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_port_driven_guide(prec):
    """The hard port on x = 0 of an open guide at 1.11 times the cut-off, 500 steps: every
    field array follows the oracle (the wave has not reached the far face)."""
    from paper_2609_16575_gb300 import gbpic

    dx = 1.0 / 20
    n, d = (240, 18, 2), (dx, dx, dx)
    dt = oracle.courant_dt(d, 0.5)
    om = 2 * np.pi
    ctx = gbpic.Context(n, d, dt, precision=prec, bc_x=1)
    ctx.set_pec(1, 1)
    ctx.set_port(1.0, om, 1.0, 1)
    F = oracle.empty_fields(n + (1,))
    guide = dict(pec_y=1, pec_z=1, port=1, e0=1.0, omega=om, tau=1.0, mode_y=1)
    done = 0
    tol = 1e-4 if prec == FP32 else 1e-11
    for k in (200, 300):
        ctx.step(k)
        oracle.run(n + (1,), d, dt, F, [], k, step0=done, guide=guide)
        done += k
        E, B, J = ctx.get_fields()
        assert rel_err(E, F[0:3]) <= tol, (done, rel_err(E, F[0:3]))
        assert rel_err(B, F[3:6]) <= tol, (done, rel_err(B, F[3:6]))
    assert np.abs(E[2]).max() > 0.5 and np.abs(E[2][:, 0, :]).max() == 0.0
    ctx.close()


def test_guide_argument_checks():
    from paper_2609_16575_gb300 import gbpic

    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=0)
    with pytest.raises(gbpic.PicError):
        c.set_port(1.0, 1.0, 1.0, 1)                  # needs an open x
    c.set_pec(1, 0)
    with pytest.raises(gbpic.PicError):                # walls act on fields only
        c.load_species_array(-1.0, 1.0, np.array([[1.5], [1.5], [1.5], [0.0], [0.0], [0.0], [1e-3]]), True)
    c.set_pec(0, 0)
    c.load_species_array(-1.0, 1.0, np.array([[1.5], [1.5], [1.5], [0.0], [0.0], [0.0], [1e-3]]), True)
    with pytest.raises(gbpic.PicError):
        c.set_pec(0, 1)
    c.close()
    c = gbpic.Context((16, 8, 8), (0.2, 0.2, 0.2), 0.05, bc_x=1)
    for bad in ((1.0, 1.0, 0.0, 1), (1.0, 1.0, 1.0, 0), (float("nan"), 1.0, 1.0, 1)):
        with pytest.raises(gbpic.PicError):
            c.set_port(*bad)
    c.close()
