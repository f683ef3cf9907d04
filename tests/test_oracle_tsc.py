"""Pins of the oracle's quadratic (TSC) particle shape (section 2.5, Eq. (16) with the
first-order cloud b1; section 5 lists higher-order shapes as an extension): the
interpolation reproduces bilinear fields exactly at every Yee stagger and adds exactly
the spline's variance 1/4 to a quadratic one; the node charge has the cloud's total,
centroid and variance; Esirkepov's deposit with this shape obeys the discrete continuity
equation exactly against that charge, carries the total current q w dX / dt, is odd
under reversal of the move, and for a move along x alone equals the closed-form charge
of the triangular cloud that crossed each plane times the transverse weights; a whole
cycle keeps Gauss's law."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W
from test_oracle_zigzag import _random_moves, _single, _wrap

# Yee staggering (cell units): component c of E sits half a cell along c, component c
# of B half a cell along the other two
HALF_E = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
HALF_B = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def _sampled(n, f):
    """E and B whose every component holds f at its own staggered sample points."""
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    E = np.empty((3, n[2], n[1], n[0]))
    B = np.empty_like(E)
    for c in range(3):
        E[c] = f(i + HALF_E[c][0], j + HALF_E[c][1], k + HALF_E[c][2])
        B[c] = f(i + HALF_B[c][0], j + HALF_B[c][1], k + HALF_B[c][2])
    return E, B


def _interior_points(rng, count, lo=5.0, hi=11.0):
    pts = [lo + rng.random(3) * (hi - lo) for _ in range(count)]
    # the nearest-sample switch points: offsets 0 and 1/2 per dimension
    pts += [np.array([7.5, 8.0, 6.5]), np.array([8.0, 7.0, 9.5]), np.array([6.25, 6.5, 7.0])]
    return pts


def test_tsc_gather_reproduces_bilinear_fields_at_every_stagger():
    n, d = (16, 16, 16), (0.2, 0.3, 0.25)
    f = lambda x, y, z: 0.3 + 1.7 * x - 0.4 * y + 2.2 * z + 0.05 * x * y - 0.03 * y * z + 0.02 * x * z
    E, B = _sampled(n, f)
    rng = np.random.default_rng(31)
    for X in _interior_points(rng, 40):
        Ep, Bp = oracle.gather(n, d, E, B, X, shape=2)
        ref = f(*X)
        np.testing.assert_allclose(np.concatenate([Ep, Bp]), ref, rtol=1e-13, atol=1e-13)


def test_tsc_gather_adds_the_spline_variance_to_quadratic_fields():
    """sum_k W2(X - k) k^2 = X^2 + 1/4 (the quadratic B-spline has variance 1/4), per
    dimension and for every stagger; a product x^2 y is separable."""
    n, d = (16, 16, 16), (0.2, 0.2, 0.2)
    rng = np.random.default_rng(32)
    pts = _interior_points(rng, 30)
    for f, ref in ((lambda x, y, z: x * x, lambda X: X[0] ** 2 + 0.25),
                   (lambda x, y, z: z * z, lambda X: X[2] ** 2 + 0.25),
                   (lambda x, y, z: x * x * y, lambda X: (X[0] ** 2 + 0.25) * X[1])):
        E, B = _sampled(n, f)
        for X in pts:
            Ep, Bp = oracle.gather(n, d, E, B, X, shape=2)
            np.testing.assert_allclose(np.concatenate([Ep, Bp]), ref(X), rtol=1e-13)


def test_tsc_charge_moments():
    """The TSC node charge of one particle: total q w, centroid X, variance 1/4 per
    dimension (cell units); 27 nodes carry it."""
    n, d = (16, 16, 16), (0.2, 0.3, 0.25)
    dV = d[0] * d[1] * d[2]
    rng = np.random.default_rng(33)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for X in _interior_points(rng, 30):
        r = oracle.rho(n, d, [_single(X, q=-1.0, w=1.3)], shape=2) * dV
        assert r.sum() == pytest.approx(-1.3, rel=1e-14)
        assert np.count_nonzero(r) <= 27
        for coord, Xc in zip((i, j, k), X):
            assert (r * coord).sum() / r.sum() == pytest.approx(Xc, rel=1e-13)
            assert (r * (coord - Xc) ** 2).sum() / r.sum() == pytest.approx(0.25, rel=1e-12)


@pytest.mark.parametrize("n,d", [((5, 6, 7), (0.2, 0.3, 0.25)), ((3, 4, 5), (1.0, 1.0, 1.0))])
def test_esirkepov_tsc_exact_continuity(n, d):
    """(rho1 - rho0)/dt + div J = 0 to round-off against the TSC charge, for moves that
    cross cell faces and the half-cell points where the nearest node changes, the ends
    of the box included."""
    rng = np.random.default_rng(34)
    dt = 0.07
    moves = _random_moves(rng, n, 200)
    moves += [(np.array([0.4, 0.6, 1.45]), np.array([0.55, 0.45, 1.55])),   # nearest node changes
              (np.array([0.5, 0.5, 0.5]), np.array([1.5, -0.5, 0.5]))]
    for X1, X2 in moves:
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.esirkepov_tsc(n, d, dt, -1.0 * 1.3, X1, X2, J)
        r0 = oracle.rho(n, d, [_single(X1)], shape=2)
        r1 = oracle.rho(n, d, [_single(_wrap(X2, n))], shape=2)
        R = oracle.continuity_residual(n, d, dt, r0, r1, J)
        scale = np.abs(J).max() / min(d) + 1.0
        assert np.abs(R).max() < 1e-13 * scale


def test_esirkepov_tsc_total_current_and_reversal():
    """sum_cells J_d dV = q w (X2_d - X1_d) d_d / dt, and the reversed move gives -J."""
    rng = np.random.default_rng(35)
    n, d, dt = (6, 5, 7), (0.2, 0.4, 0.3), 0.05
    dV = d[0] * d[1] * d[2]
    for X1, X2 in _random_moves(rng, n, 100):
        J = np.zeros((3, n[2], n[1], n[0]))
        oracle.esirkepov_tsc(n, d, dt, 0.7, X1, X2, J)
        for c in range(3):
            np.testing.assert_allclose(J[c].sum() * dV, 0.7 * (X2[c] - X1[c]) * d[c] / dt, rtol=1e-12, atol=1e-14)
        # the reversed move, expressed from the end point's own cell
        Jr = np.zeros_like(J)
        oracle.esirkepov_tsc(n, d, dt, 0.7, X2, X1, Jr)
        np.testing.assert_allclose(Jr, -J, rtol=0, atol=1e-13 * np.abs(J).max())


def _cloud_cdf(t):
    """Charge of the triangular cloud b1 (1 - |t| on |t| <= 1) below t: its cumulative."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t <= -1.0, 0.0, 1.0)
    out = np.where((t > -1.0) & (t <= 0.0), 0.5 * (1.0 + t) ** 2, out)
    out = np.where((t > 0.0) & (t < 1.0), 1.0 - 0.5 * (1.0 - t) ** 2, out)
    return out


def _w2(r):
    r = np.abs(r)
    return np.where(r <= 0.5, 0.75 - r * r, np.where(r < 1.5, 0.5 * (1.5 - r) ** 2, 0.0))


def test_esirkepov_tsc_move_along_x_is_the_cloud_flux():
    """A move along x alone: Jy = Jz = 0 and Jx(i+1/2, j, k) dt dy dz / (q w) =
    [T(X2 - i - 1/2) - T(X1 - i - 1/2)] W2(Y - j) W2(Z - k), T the cumulative charge of
    the triangular cloud b1: the part of the cloud that crossed the plane x = i + 1/2."""
    n, d, dt, qw = (16, 16, 16), (0.2, 0.3, 0.25), 0.04, 0.9
    rng = np.random.default_rng(36)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for _ in range(40):
        X1 = 5.0 + rng.random(3) * 6.0
        X2 = X1.copy()
        X2[0] += (rng.random() * 2 - 1) * 0.95
        J = np.zeros((3,) + n[::-1])
        oracle.esirkepov_tsc(n, d, dt, qw, X1, X2, J)
        assert np.abs(J[1]).max() == 0.0 and np.abs(J[2]).max() == 0.0
        ref = (_cloud_cdf(X2[0] - i - 0.5) - _cloud_cdf(X1[0] - i - 0.5)) * _w2(X1[1] - j) * _w2(X1[2] - k)
        ref *= qw / (dt * d[1] * d[2])
        np.testing.assert_allclose(J[0], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_tsc_cycle_keeps_gauss_law():
    """Twenty cycles of a warm plasma with the TSC shape: G = div E - rho - rho_ion with
    the TSC charge keeps its initial value (continuity plus Yee, section 2.3)."""
    wl = W.thermal((8, 6, 10), 0.2, 8, 0.08, seed=77, steps=20)
    n, d, dt = wl.n, wl.d, wl.dt
    sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
    F = oracle.empty_fields(n)

    def gauss():
        return oracle.divergence(n, d, F[0:3]) - oracle.rho(n, d, sp, rho_ion=1.0, shape=2)

    G0 = gauss()
    rho_max = np.abs(oracle.rho(n, d, sp, shape=2)).max()
    oracle.run(n, d, dt, F, sp, 20, guide={"shape": 2})
    assert np.abs(F[6:9]).max() > 0
    assert np.abs(gauss() - G0).max() < 1e-12 * rho_max


def test_tsc_cycle_differs_from_cic_and_conserves_energy():
    """The shape option changes the run (the TSC path is taken), and a warm plasma's
    total energy U_E + U_B + K stays within 1 % over 100 cycles."""
    wl = W.thermal((8, 8, 8), 0.2, 8, 0.05, seed=78, steps=100)
    n, d, dt = wl.n, wl.d, wl.dt
    runs = {}
    for shape in (1, 2):
        sp = [oracle.Species(s.q, s.m, s.P) for s in wl.species]
        F = oracle.empty_fields(n)
        h = oracle.run(n, d, dt, F, sp, 100, guide={"shape": shape})
        runs[shape] = (h, sp[0].P)
    h = runs[2][0]
    tot = h.sum(axis=1)
    assert np.abs(tot / tot[0] - 1).max() < 0.01
    assert np.abs(runs[1][1] - runs[2][1]).max() > 1e-6
