"""Pins of the oracle's charge-conserving zigzag deposit (section 2.5) by invariants
that do not depend on the deposit formula: exact discrete continuity (Eq. (12)),
total current, uniqueness in one dimension and antisymmetry."""
import numpy as np
import pytest

import oracle


def _single(X, q=-1.0, w=1.3):
    P = np.zeros((7, 1))
    P[0:3, 0] = X
    P[6, 0] = w
    return oracle.Species(q, 1.0, P)


def _wrap(X, n):
    return np.array([x % m for x, m in zip(X, n)])


def _random_moves(rng, n, count, max_step=0.9):
    out = []
    for _ in range(count):
        X1 = rng.random(3) * np.array(n)
        D = (rng.random(3) * 2 - 1) * max_step
        X2 = X1 + D
        # keep |floor(X2) - floor(X1)| <= 1 per dimension (one cell per step)
        for dd in range(3):
            if abs(np.floor(X2[dd]) - np.floor(X1[dd])) > 1:
                X2[dd] = X1[dd]
        out.append((X1, X2))
    # moves that end exactly on faces, edges and corners, and wrap the box
    out.append((np.array([0.25, 0.5, 0.75]), np.array([1.0, 0.5, 0.75])))
    out.append((np.array([0.6, 0.7, 0.8]), np.array([1.0, 1.0, 1.0])))
    out.append((np.array([0.1, 0.2, 0.3]), np.array([-0.2, -0.1, -0.05])))
    out.append((np.array([n[0] - 0.1, n[1] - 0.3, 0.2]), np.array([n[0] + 0.15, n[1] + 0.1, -0.1])))
    return out


@pytest.mark.parametrize("n,d", [((3, 4, 5), (0.2, 0.3, 0.25)), ((1, 2, 3), (1.0, 1.0, 1.0))])
def test_zigzag_exact_continuity(n, d):
    """rho from CIC before and after the move and the deposited J satisfy
    (rho1 - rho0)/dt + div J = 0 to round-off, for moves crossing 0..3 faces."""
    rng = np.random.default_rng(11)
    dt = 0.07
    for X1, X2 in _random_moves(rng, n, 200):
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.zigzag(n, d, dt, -1.0 * 1.3, X1, X2, J)
        r0 = oracle.rho(n, d, [_single(X1)])
        r1 = oracle.rho(n, d, [_single(_wrap(X2, n))])
        R = oracle.continuity_residual(n, d, dt, r0, r1, J)
        scale = np.abs(J).max() / min(d) + 1.0
        assert np.abs(R).max() < 1e-13 * scale


def test_zigzag_total_current():
    """sum_cells J_d dV = q w (X2_d - X1_d) d_d / dt for each component."""
    rng = np.random.default_rng(12)
    n, d, dt = (4, 3, 5), (0.2, 0.4, 0.3), 0.05
    for X1, X2 in _random_moves(rng, n, 100):
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.zigzag(n, d, dt, 0.8, X1, X2, J)
        dV = np.prod(d)
        for c in range(3):
            assert abs(J[c].sum() * dV - 0.8 * (X2[c] - X1[c]) * d[c] / dt) < 1e-13


def test_zigzag_one_dimensional_is_unique():
    """For a move along x only, continuity plus the total current fix J_x uniquely:
    J_x(i+1/2) = J0 - (dx/dt) sum_{i' <= i} (rho1 - rho0)(i') summed cumulatively.
    Built here by brute force from the CIC charges alone."""
    rng = np.random.default_rng(13)
    n, d, dt = (7, 1, 1), (0.3, 1.0, 1.0), 0.1
    for _ in range(100):
        X1 = np.array([rng.random() * 7, 0.4, 0.6])
        X2 = X1 + np.array([(rng.random() * 2 - 1) * 0.95, 0, 0])
        if abs(np.floor(X2[0]) - np.floor(X1[0])) > 1:
            continue
        J = np.zeros((3, 1, 1, 7))
        oracle.zigzag(n, d, dt, 1.0, X1, X2, J)
        r0 = oracle.rho(n, d, [_single(X1, q=1.0, w=1.0)])[0, 0]
        r1 = oracle.rho(n, d, [_single(_wrap(X2, n), q=1.0, w=1.0)])[0, 0]
        flux = -np.cumsum(r1 - r0) * d[0] / dt          # J(i+1/2) - J(-1/2)
        total = 1.0 * (X2[0] - X1[0]) * d[0] / dt / np.prod(d)
        J0 = (total - flux.sum()) / 7.0
        assert np.abs(J[0, 0, 0] - (J0 + flux)).max() < 1e-12
        assert np.abs(J[1:]).max() < 1e-15


def test_zigzag_antisymmetric_under_reversal():
    """The reversed move deposits exactly the opposite current."""
    rng = np.random.default_rng(14)
    n, d, dt = (3, 3, 3), (0.2, 0.2, 0.2), 0.05
    for X1, X2 in _random_moves(rng, n, 60):
        J1 = np.zeros((3, 3, 3, 3))
        J2 = np.zeros((3, 3, 3, 3))
        oracle.zigzag(n, d, dt, 1.0, X1, X2, J1)
        # reverse from the wrapped end point back to the unwrapped start
        X2w = _wrap(X2, n)
        oracle.zigzag(n, d, dt, 1.0, X2w, X1 + (X2w - X2), J2)
        assert np.abs(J1 + J2).max() < 1e-12 * (np.abs(J1).max() + 1)


def test_midpoint_product_alone_violates_3d_continuity():
    """The reading behind the Dy Dz / 12 term: without it a diagonal move inside one
    cell leaves a continuity residual of (Dx Dy Dz / 4) per segment (brute force,
    numpy only), so the plain product of midpoint weights is not charge conserving
    in three dimensions."""
    n, d, dt = (2, 2, 2), (1.0, 1.0, 1.0), 1.0
    X1 = np.array([0.2, 0.2, 0.2])
    X2 = np.array([0.6, 0.6, 0.6])
    D = X2 - X1
    mid = (X1 + X2) / 2
    J = np.zeros((3, 2, 2, 2))
    for comp in range(3):
        p, r = (comp + 1) % 3, (comp + 2) % 3
        for b in range(2):
            for c in range(2):
                idx = [0, 0, 0]
                idx[p] += b
                idx[r] += c
                wp = mid[p] if b else 1 - mid[p]
                wr = mid[r] if c else 1 - mid[r]
                J[comp, idx[2], idx[1], idx[0]] += D[comp] * wp * wr
    r0 = oracle.rho(n, d, [_single(X1, q=1.0, w=1.0)])
    r1 = oracle.rho(n, d, [_single(X2, q=1.0, w=1.0)])
    R = oracle.continuity_residual(n, d, dt, r0, r1, J)
    # single straight segment: residual magnitude Dx Dy Dz / 4 at the corner nodes
    assert abs(abs(R[0, 0, 0]) - np.prod(D) / 4) < 1e-14
    # the oracle's deposit of the same move (two segments, with the term) is exact
    J2 = np.zeros((3, 2, 2, 2))
    oracle.zigzag(n, d, dt, 1.0, X1, X2, J2)
    assert np.abs(oracle.continuity_residual(n, d, dt, r0, r1, J2)).max() < 1e-14
