"""Pins of the oracle's staggered CIC gather (section 2.5) and the momentum
back-push (section 2.4) by exactness on linear fields and time reversibility."""
import numpy as np

import oracle

HALF_E = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
HALF_B = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def test_gather_exact_on_linear_fields():
    """Trilinear interpolation reproduces a field that is linear in space exactly,
    provided each component is sampled at its own Yee location: a half-cell error in
    the staggering of any component shows up as an offset of half its gradient."""
    rng = np.random.default_rng(21)
    n, d = (8, 9, 10), (0.2, 0.3, 0.25)
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    a = rng.standard_normal((6, 4))
    F = np.zeros((6, n[2], n[1], n[0]))
    for c in range(6):
        h = HALF_E[c] if c < 3 else HALF_B[c - 3]
        F[c] = a[c, 0] + a[c, 1] * (ii + h[0]) + a[c, 2] * (jj + h[1]) + a[c, 3] * (kk + h[2])
    for _ in range(300):
        # stay two cells away from the periodic seam, where the field is not linear
        X = np.array([2 + rng.random() * (n[0] - 4), 2 + rng.random() * (n[1] - 4), 2 + rng.random() * (n[2] - 4)])
        Ep, Bp = oracle.gather(n, d, np.ascontiguousarray(F[0:3]), np.ascontiguousarray(F[3:6]), X)
        expect = a[:, 0] + a[:, 1] * X[0] + a[:, 2] * X[1] + a[:, 3] * X[2]
        assert np.abs(np.r_[Ep, Bp] - expect).max() < 1e-12


def test_gather_partition_of_unity_and_tie():
    """A uniform field is returned unchanged anywhere, including on the half-cell tie."""
    n, d = (3, 3, 3), (1.0, 1.0, 1.0)
    E = np.ones((3, 3, 3, 3)) * np.array([1.0, -2.0, 3.0])[:, None, None, None]
    B = np.ones((3, 3, 3, 3)) * np.array([0.5, 0.25, -4.0])[:, None, None, None]
    for X in ([0.5, 0.5, 0.5], [0.0, 0.0, 0.0], [2.999999, 1.5, 0.25]):
        Ep, Bp = oracle.gather(n, d, E, B, np.array(X))
        assert np.allclose(Ep, [1, -2, 3], atol=1e-14) and np.allclose(Bp, [0.5, 0.25, -4], atol=1e-14)


def test_backpush_is_reversible():
    """The back-push u^0 -> u^{-1/2} is a Boris step of -dt/2; a forward Boris step of
    +dt/2 in the same fields returns u^0 (the Boris map is time reversible)."""
    rng = np.random.default_rng(22)
    n, d = (4, 4, 4), (0.5, 0.5, 0.5)
    dt = 0.1
    E = np.ones((3, 4, 4, 4)) * np.array([0.3, -0.2, 0.1])[:, None, None, None]
    B = np.ones((3, 4, 4, 4)) * np.array([0.0, 0.4, 1.1])[:, None, None, None]
    P = np.zeros((7, 20))
    P[0:3] = rng.random((3, 20)) * 4
    P[3:6] = rng.standard_normal((3, 20)) * 0.5
    P[6] = 1.0
    sp = oracle.Species(-1.0, 1.0, P.copy())
    oracle.backpush(n, d, dt, E, B, sp)       # uniform fields: curl E = 0, so B^0 = B^{-1/2}
    for p in range(20):
        u = oracle.boris(-1.0 * (dt / 2) / 2.0, [0.3, -0.2, 0.1], [0.0, 0.4, 1.1], sp.P[3:6, p])
        assert np.abs(u - P[3:6, p]).max() < 1e-14
