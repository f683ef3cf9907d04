"""Pins of the oracle's moving window (section 2.2: an operation at the end of the cycle;
section 4: the laser-wakefield run moves its window along the laser).  The window
moves one cell along +x; fields and particles shift with it, the first column leaves
and the last column receives fresh plasma at rest.

While nothing reaches its edges, a moving window is exactly a sub-box of a fixed box
that is long enough: the same cycles act on the same values, only the cell indices
differ by the number of moves.  These tests pin the shift, the removal and the
injection of the oracle against a fixed-box run of the same oracle and against the
initial plasma loading, which share none of the window code."""
import numpy as np

import oracle

D = (0.1, 0.15, 0.15)
DT = oracle.courant_dt(D, 0.5)
PROFILE = dict(density=0.5, x0=-10.0, ramp=30.0)


def _plasma(nx, ny, nz, origin, ppd=2, density=0.5, x0=-10.0, ramp=30.0):
    """A ppd^3 lattice per cell at rest, density density * clip((x - x0) / ramp, 0, 1)
    at absolute x = origin + window x (cell units); no particle where it is zero."""
    off = (2 * np.arange(ppd) + 1) / (2.0 * ppd)
    xs = (np.arange(nx)[:, None] + off[None, :]).ravel()
    X = (np.arange(nx)[:, None] + origin + off[None, :]).ravel()
    prof = density * np.clip((X - x0) / ramp, 0.0, 1.0)
    w = prof * D[0] * D[1] * D[2] / ppd ** 3
    ys = (np.arange(ny)[:, None] + off).ravel()
    zs = (np.arange(nz)[:, None] + off).ravel()
    Zg, Yg, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    Wg = np.broadcast_to(w[None, None, :], Xg.shape)
    keep = Wg.ravel() > 0
    zero = np.zeros(keep.sum())
    return np.stack([Xg.ravel()[keep], Yg.ravel()[keep], Zg.ravel()[keep], zero, zero, zero, Wg.ravel()[keep]])


def _pulse(nx, ny, nz, xc, half_width=4.0, amplitude=0.5, wavelength=4.0):
    """A y-polarised pulse travelling along +x with compact support |x - xc| < half_width
    (cells): Ey on the x nodes at t = 0, Bz at x + 1/2 at t = -dt/2."""
    F = oracle.empty_fields((nx, ny, nz, 1))

    def f(x):
        r = x - xc
        inside = np.abs(r) < half_width
        return np.where(inside, amplitude * np.sin(2 * np.pi * r / wavelength)
                        * np.cos(np.pi * r / (2 * half_width)) ** 2, 0.0)

    x = np.arange(nx + 1, dtype=np.float64)
    F[1] = f(x)[None, None, :]
    F[5, :, :, :nx] = f(x[:nx] + 0.5 + 0.5 * DT / D[0])[None, None, :]
    return F


def _window(every=2, start=0):
    return dict(start=start, every=every, species=0, ppc=(2, 2, 2), **PROFILE)


def _sorted(C, Q):
    order = np.lexsort((Q[2], Q[1], Q[0], C[2], C[1], C[0]))
    return C[:, order], Q[:, order]


def test_moves_schedule():
    """A move ends every `every`-th cycle from `start` on; the count before a cycle
    agrees with the moves of the cycles before it."""
    w = _window(every=3, start=5)
    moves = [s for s in range(40) if oracle.window_moves_after(w, s)]
    assert moves[:3] == [7, 10, 13]
    for s in range(40):
        assert oracle.window_moves_before(w, s) == sum(1 for m in moves if m < s)


def test_window_is_a_moving_subbox():
    """A pulse in a plasma with a density ramp, 12 cycles, a move every 2 cycles: the
    window's fields, current and particles equal those of a fixed 96-cell box on the
    cells the window covers, exactly (the field support grows one cell per cycle and
    stays clear of the window's faces; the particles outside it are at rest)."""
    ny = nz = 4
    nw, nb, steps = 64, 96, 12
    win = _window()
    Fw = _pulse(nw, ny, nz, 40.0)
    Fb = _pulse(nb, ny, nz, 40.0)
    sw = [oracle.Species(-1.0, 1.0, _plasma(nw, ny, nz, 0))]
    sb = [oracle.Species(-1.0, 1.0, _plasma(nb, ny, nz, 0))]
    n0 = sw[0].n
    oracle.run_window((nw, ny, nz, 1), D, DT, Fw, sw, steps, win)
    oracle.run((nb, ny, nz, 1), D, DT, Fb, sb, steps)
    origin = oracle.window_moves_before(win, steps)
    assert origin == 6
    # the big box's fields stay clear of the window's edges (the precondition)
    support = np.nonzero(np.abs(Fb).max(axis=(0, 1, 2)) > 0)[0]
    assert support.min() > origin + 2 and support.max() < nw - 2
    assert np.array_equal(Fw[0:6], Fb[0:6][..., origin:origin + nw + 1])
    # J is that of the last cycle, before its move
    assert np.array_equal(Fw[6:9], Fb[6:9][..., origin - 1:origin + nw])
    assert np.abs(Fw[6:9]).max() > 0
    # particles: the window's (alive) ones are the big box's on cells origin .. origin+nw-1
    s, b = sw[0], sb[0]
    alive_w = s.Q[6] > 0
    inside_b = (b.C[0] >= origin) & (b.C[0] < origin + nw)
    Cw, Qw = _sorted(s.C[:, alive_w] + np.array([[origin], [0], [0]]), s.Q[:, alive_w])
    Cb, Qb = _sorted(b.C[:, inside_b], b.Q[:, inside_b])
    assert Cw.shape == Cb.shape
    assert np.array_equal(Cw, Cb) and np.array_equal(Qw, Qb)
    assert np.abs(Qw[3:6]).max() > 1e-3           # the pulse moved electrons
    assert s.n > n0 and (~alive_w).sum() > 0       # plasma came in and left


def test_injected_plasma_is_the_loaded_plasma_of_the_moved_box():
    """Without fields nothing moves: after 9 moves the window holds exactly the plasma
    that loading a box at absolute x = 9 gives, the ramp included."""
    nw, ny, nz = 16, 2, 2
    win = _window(every=1, start=3)
    win["x0"], win["ramp"] = 14.0, 6.0
    F = oracle.empty_fields((nw, ny, nz, 1))
    s = oracle.Species(-1.0, 1.0, _plasma(nw, ny, nz, 0, x0=14.0, ramp=6.0))
    oracle.run_window((nw, ny, nz, 1), D, DT, F, [s], 12, win)
    origin = oracle.window_moves_before(win, 12)
    assert origin == 9
    ref = oracle.Species(-1.0, 1.0, _plasma(nw, ny, nz, origin, x0=14.0, ramp=6.0))
    alive = s.Q[6] > 0
    Cw, Qw = _sorted(s.C[:, alive], s.Q[:, alive])
    Cr, Qr = _sorted(ref.C, ref.Q)
    assert np.array_equal(Cw, Cr) and np.array_equal(Qw, Qr)
    assert np.abs(F).max() == 0.0


def test_window_plasma_order_and_weights():
    """The new column's plasma: ordered z cell, y cell, z offset, y offset, x offset,
    at rest, weights from the ramp at the particles' absolute x (none in vacuum)."""
    win = dict(start=0, every=1, species=0, ppc=(4, 1, 2), density=2.0, x0=10.5, ramp=4.0)
    n = (8, 3, 2)
    P = oracle.window_plasma(n, D, win, origin=3)    # last column: absolute x = 10 .. 11
    # x offsets 1/8, 3/8, 5/8, 7/8 at absolute 10.125 ... 10.875: only 10.625, 10.875 are past x0
    assert P.shape == (7, 2 * 3 * 2 * 1 * 2)
    assert np.allclose(P[0, :2], [7.625, 7.875]) and np.all(P[3:6] == 0)
    np.testing.assert_allclose(P[6, :2], 2.0 * np.array([0.125, 0.375]) / 4.0 * D[0] * D[1] * D[2] / 8,
                               rtol=1e-15)
    assert np.allclose(P[2, :4], [0.25, 0.25, 0.75, 0.75])   # z offset before y cell changes
    assert np.allclose(P[1, 4:8], [1.5, 1.5, 1.5, 1.5])


def test_lwfa_window_continues_the_loaded_plasma():
    """The laser-wakefield workload's window brings in exactly the plasma that its loader
    puts in the same absolute cells of a longer box (lattice, ramp and weights), and moves
    no faster than light."""
    from paper_2609_16575_gb300 import workloads as W

    n = (24, 4, 4)                                     # new columns at x = 24 .. 62 cross the ramp 20 .. 50
    kw = dict(ppc_per_dim=2, density=0.01, x0=20, ramp=30)
    wl = W.lwfa(n=n, window_start=0, **kw)
    win = wl.window.as_dict()
    assert win["every"] * wl.dt >= wl.d[0]
    long_box = W.lwfa(n=(n[0] + 40, n[1], n[2]), **kw).species[0].P
    for origin in (1, 13, 27, 39):
        new = oracle.window_plasma(n, wl.d, win, origin)
        col = origin + n[0] - 1                        # the new column's absolute x
        ref = long_box[:, (long_box[0] >= col) & (long_box[0] < col + 1)].copy()
        ref[0] -= origin                               # into window coordinates
        a = new[:, np.lexsort(new[::-1])]
        b = ref[:, np.lexsort(ref[::-1])]
        assert a.shape == b.shape, (origin, a.shape, b.shape)
        np.testing.assert_array_equal(a, b)
