"""Pins of the oracle's Esirkepov deposit (Esirkepov 2001; section 2.5 names it among the
charge-conserving schemes, next to the ZigZag the paper uses) with the CIC shape:
exact discrete continuity against the independent CIC charge, the total current, equality
with the pinned ZigZag for moves inside one cell (where both are the exact flux of a
straight segment through the trilinear cloud), and a whole cycle that keeps Gauss's law."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from test_oracle_zigzag import _random_moves, _single, _wrap


@pytest.mark.parametrize("n,d", [((3, 4, 5), (0.2, 0.3, 0.25)), ((1, 2, 3), (1.0, 1.0, 1.0))])
def test_esirkepov_exact_continuity(n, d):
    """(rho1 - rho0)/dt + div J = 0 to round-off for moves crossing 0..3 faces, the
    ends of the box and cell corners included."""
    rng = np.random.default_rng(21)
    dt = 0.07
    for X1, X2 in _random_moves(rng, n, 200):
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.esirkepov(n, d, dt, -1.0 * 1.3, X1, X2, J)
        r0 = oracle.rho(n, d, [_single(X1)])
        r1 = oracle.rho(n, d, [_single(_wrap(X2, n))])
        R = oracle.continuity_residual(n, d, dt, r0, r1, J)
        scale = np.abs(J).max() / min(d) + 1.0
        assert np.abs(R).max() < 1e-13 * scale


def test_esirkepov_total_current():
    """sum_cells J_d dV = q w (X2_d - X1_d) d_d / dt for each component."""
    rng = np.random.default_rng(22)
    n, d, dt = (4, 3, 5), (0.2, 0.4, 0.3), 0.05
    dV = d[0] * d[1] * d[2]
    for X1, X2 in _random_moves(rng, n, 100):
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.esirkepov(n, d, dt, 0.7, X1, X2, J)
        for c in range(3):
            np.testing.assert_allclose(J[c].sum() * dV, 0.7 * (X2[c] - X1[c]) * d[c] / dt, rtol=1e-12, atol=1e-14)


def test_equal_to_zigzag_inside_a_cell_and_not_across():
    """Inside one cell both schemes give the exact flux of the straight segment; across
    cell faces ZigZag relays through a face point and the two differ (both conserve)."""
    rng = np.random.default_rng(23)
    n, d, dt = (4, 4, 4), (0.2, 0.25, 0.3), 0.05
    differ = 0
    for X1, X2 in _random_moves(rng, n, 300):
        Je = np.zeros((3, 4, 4, 4))
        Jz = np.zeros((3, 4, 4, 4))
        oracle.esirkepov(n, d, dt, 1.1, X1, X2, Je)
        oracle.zigzag(n, d, dt, 1.1, X1, X2, Jz)
        inside = np.all(np.floor(X1) == np.floor(X2))
        err = np.abs(Je - Jz).max() / (np.abs(Jz).max() + 1e-300)
        if inside:
            assert err < 1e-13, err
        elif np.sum(np.floor(X1) != np.floor(X2)) >= 2:
            differ += err > 1e-6
    assert differ > 20


def test_cycle_with_esirkepov_keeps_gauss():
    """A hot periodic plasma for 20 cycles with the Esirkepov deposit: div E - rho
    stays at its initial value to round-off."""
    wl = W.thermal((6, 6, 6), 0.2, 4, 0.4, seed=24)
    n, d, dt = wl.n, wl.d, wl.dt
    sp = [oracle.Species(-1.0, 1.0, wl.species[0].P)]
    F = oracle.empty_fields(n)
    g0 = oracle.divergence(n, d, F[0:3]) - oracle.rho(n, d, sp, wl.rho_ion)
    oracle.run(n, d, dt, F, sp, 20, guide=dict(esirkepov=1))
    g1 = oracle.divergence(n, d, F[0:3]) - oracle.rho(n, d, sp, wl.rho_ion)
    assert np.abs(g1 - g0).max() < 1e-12 * np.abs(oracle.rho(n, d, sp)).max()
    assert np.abs(F[6:9]).max() > 0
