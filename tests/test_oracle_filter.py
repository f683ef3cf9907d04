"""Pins of the oracle's compensated binomial current filter (section 2.2 counts
"compensated smoothing" among the operations of a cycle, section 2.6 a current-filtering
module; the paper gives no scheme and its runs use none).  Reading: per dimension one
convolution with p binomial stencils (1/4, 1/2, 1/4) and the compensator
(-p/4, 1 + p/2, -p/4).  On a periodic grid a Fourier mode is an eigenvector of it with
eigenvalue prod_d (1 - s_d)^p (1 + p s_d), s_d = sin^2(k_d d_d / 2), which these tests
check against the closed form."""
import numpy as np
import pytest

import oracle
from paper_2609_16575_gb300 import workloads as W


def _mode_field(n, m, phase):
    """cos(2 pi sum_d m_d i_d / n_d + phase) on the cell indices of a (nz, ny, nx) grid."""
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return np.cos(2 * np.pi * (m[0] * ii / n[0] + m[1] * jj / n[1] + m[2] * kk / n[2]) + phase)


def _transfer(n, m, passes, compensate):
    T = 1.0
    for dd in range(3):
        s = np.sin(np.pi * m[dd] / n[dd]) ** 2
        T *= (1 - s) ** passes * ((1 + passes * s) if compensate else 1.0)
    return T


@pytest.mark.parametrize("passes,compensate", [(1, False), (1, True), (2, True), (3, False), (4, True)])
def test_fourier_modes_are_scaled_by_the_transfer_function(passes, compensate):
    n, d = (12, 10, 8), (0.2, 0.3, 0.25)
    for m in ((1, 0, 0), (0, 3, 1), (5, 2, 3), (6, 0, 0), (2, 5, 4)):
        J = np.zeros((3, n[2], n[1], n[0]))
        for c in range(3):
            J[c] = _mode_field(n, m, 0.3 + c)
        ref = J * _transfer(n, m, passes, compensate)
        oracle.current_filter(n, d, J, passes, compensate)
        assert np.abs(J - ref).max() <= 1e-14, (m, np.abs(J - ref).max())


def test_nyquist_removed_and_long_waves_kept():
    """The binomial kernel removes the grid-scale mode; the compensated one keeps a long
    wave to fourth order in k (1 - s^2 per dimension)."""
    n, d = (16, 4, 4), (0.1, 0.1, 0.1)
    J = np.zeros((3, 4, 4, 16))
    J[0] = _mode_field(n, (8, 0, 0), 0.0)
    oracle.current_filter(n, d, J, 1, False)
    assert np.abs(J).max() <= 1e-15
    J[1] = _mode_field(n, (1, 0, 0), 0.7)
    ref = J[1].copy()
    oracle.current_filter(n, d, J, 1, True)
    s = np.sin(np.pi / 16) ** 2
    np.testing.assert_allclose(J[1], ref * (1 - s * s), atol=1e-15)


def test_total_current_is_kept_on_a_periodic_grid():
    rng = np.random.Generator(np.random.PCG64(81))
    n, d = (9, 7, 5), (0.2, 0.2, 0.2)
    J = rng.standard_normal((3, 5, 7, 9))
    tot = J.sum(axis=(1, 2, 3))
    oracle.current_filter(n, d, J, 2, True)
    np.testing.assert_allclose(J.sum(axis=(1, 2, 3)), tot, atol=1e-12)


def test_open_x_is_local_and_drops_what_leaves():
    """Along an open x: a current far from the faces is filtered as on the periodic grid;
    a current on the first plane keeps only the kernel's weights that land inside (3/4 of
    a single binomial pass), and the face plane x = nx is left alone."""
    rng = np.random.Generator(np.random.PCG64(82))
    n, d = (20, 6, 6), (0.2, 0.2, 0.2)
    Jp = np.zeros((3, 6, 6, 20))
    Jp[:, :, :, 8:12] = rng.standard_normal((3, 6, 6, 4))
    Jo = np.zeros((3, 6, 6, 21))
    Jo[..., :20] = Jp
    oracle.current_filter(n, d, Jp, 2, True)
    oracle.current_filter(n + (1,), d, Jo, 2, True)
    np.testing.assert_allclose(Jo[..., :20], Jp, atol=1e-15)
    J = np.zeros((3, 6, 6, 21))
    J[1, :, :, 0] = 1.0
    J[2, :, :, 20] = 5.0
    oracle.current_filter(n + (1,), d, J, 1, False)
    np.testing.assert_allclose(J[1].sum(axis=2), 0.75, atol=1e-15)
    np.testing.assert_allclose(J[1, :, :, 0:2], np.broadcast_to([0.5, 0.25], (6, 6, 2)), atol=1e-15)
    assert np.all(J[2, :, :, 20] == 5.0)


def test_filter_acts_on_the_deposit_before_ampere():
    """One cycle from zero fields: E^1 = -dt J^{1/2} with J the filtered deposit, and the
    filtered cycle's J is the filter applied to the unfiltered cycle's J."""
    wl = W.thermal((8, 8, 8), 0.2, 2, 0.3, seed=83)
    filt = (1, 1)
    F0 = oracle.empty_fields(wl.n)
    F1 = oracle.empty_fields(wl.n)
    s0 = [oracle.Species(-1.0, 1.0, wl.species[0].P)]
    s1 = [oracle.Species(-1.0, 1.0, wl.species[0].P)]
    oracle.run(wl.n, wl.d, wl.dt, F0, s0, 1)
    oracle.run(wl.n, wl.d, wl.dt, F1, s1, 1, current_filter=filt)
    Jf = F0[6:9].copy()
    oracle.current_filter(wl.n, wl.d, Jf, *filt)
    np.testing.assert_allclose(F1[6:9], Jf, rtol=0, atol=1e-15 * np.abs(Jf).max())
    np.testing.assert_allclose(F1[0:3], -wl.dt * F1[6:9], rtol=0, atol=1e-15 * np.abs(F1[0:3]).max())
    assert np.abs(F1[6:9] - F0[6:9]).max() > 1e-3 * np.abs(F0[6:9]).max()
