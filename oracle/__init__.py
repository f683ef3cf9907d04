"""Plain FP64 CPU oracle of the explicit EM-PIC cycle (KEMPIC-3D, arxiv 2609.16575).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2609_16575_gb300``) never does, and the two share no code.

The arithmetic lives in ``pic_oracle.c`` (plain C, FP64, one loop per
operation).  This module compiles it with gcc, loads it with ctypes and adds
numpy helpers.  It also holds two closed forms that the tests use as pins and
inputs: the Yee vacuum eigenmode (``plane_wave``) and the discrete cold-plasma
frequency of a two-sheets-per-cell lattice (``cold_plasma_omega``).

Array conventions (see the header of ``pic_oracle.c``): a field set is a
``(9, nz, ny, nx)`` float64 array holding Ex Ey Ez Bx By Bz Jx Jy Jz at their
Yee locations; a species is given as a ``(7, np)`` float64 array holding X Y Z
(cell units), ux uy uz and w, and kept internally as integer cells plus in-cell
offsets.

Parity status of every function: pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants and the paper's printed values, except where a
docstring says "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile ``pic_oracle.c`` into ``_build/liboracle.so`` (FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.or_faraday.argtypes = [_ip, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double]
            L.or_ampere.argtypes = [_ip, _dp, ctypes.c_double, _dp, _dp, _dp]
            L.or_gather.argtypes = [_ip, _dp, _dp, _dp, _dp, _dp, _dp]
            L.or_boris.argtypes = [ctypes.c_double, _dp, _dp, _dp]
            L.or_boris_orbit.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                         ctypes.c_long, ctypes.c_int, _dp, _dp]
            L.or_zigzag.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            L.or_rho.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_long, _dp, _dp, _dp]
            L.or_rho_tsc.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_long, _dp, _dp, _dp]
            L.or_divergence.argtypes = [_ip, _dp, _dp, _dp]
            L.or_divergence_b.argtypes = [_ip, _dp, _dp, _dp]
            L.or_backpush.argtypes = [_ip, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_long, _dp, _dp, ctypes.c_int]
            L.or_step.argtypes = [_ip, _dp, ctypes.c_double, _dp, ctypes.c_int, _dp, _lp,
                                  ctypes.POINTER(_dp), ctypes.POINTER(_dp), _dp, ctypes.c_long, _dp, _dp, _dp]
            L.or_run.argtypes = [_ip, _dp, ctypes.c_double, _dp, ctypes.c_int, _dp, _lp,
                                 ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.c_long, _dp, ctypes.c_long, _dp, _dp,
                                 _dp]
            L.or_current_filter.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int]
            L.or_esirkepov.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            L.or_esirkepov_tsc.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            L.or_gather_tsc.argtypes = [_ip, _dp, _dp, _dp, _dp, _dp, _dp]
            L.or_push.argtypes = [_ip, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                  _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
            L.or_push.restype = ctypes.c_double
            L.or_window_shift.argtypes = [_ip, _dp, _dp, ctypes.c_int, _lp, ctypes.POINTER(_dp), ctypes.POINTER(_dp)]
            L.or_gauss_x.argtypes = [_ip, _dp, _dp, _dp]
            L.or_gauss_x.restype = ctypes.c_double
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _grid(n, d):
    """n = (nx, ny, nz) for a periodic box, or (nx, ny, nz, 1) for an open x dimension."""
    n = list(n) + [0] * (4 - len(n))
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.float64)
    return n, d, n.ctypes.data_as(_ip), _p(d)


def field_shape(n):
    """(nz, ny, values per x line): nx, or nx + 1 nodes with an open x dimension."""
    open_x = len(n) > 3 and n[3]
    return (int(n[2]), int(n[1]), int(n[0]) + (1 if open_x else 0))


class Species:
    """One particle species for the oracle: charge ``q`` and mass ``m`` per physical
    particle.  Given as a ``(7, np)`` array (X, Y, Z in cell units; ux, uy, uz; w), it is
    held as integer cells ``C`` (3, np) and ``Q`` (7, np: in-cell offsets, momenta,
    weights), so that FP64 resolves 2^-53 of a cell anywhere in the box.  ``P`` returns
    the 7-row form again (positions rounded to FP64 only there)."""

    def __init__(self, q: float, m: float, P: np.ndarray):
        self.q = float(q)
        self.m = float(m)
        P = np.asarray(P, dtype=np.float64)
        assert P.ndim == 2 and P.shape[0] == 7
        self.C = np.ascontiguousarray(np.floor(P[0:3]))
        self.Q = np.ascontiguousarray(P.copy())
        self.Q[0:3] = P[0:3] - self.C
        up = self.Q[0:3] >= 1.0            # a rounded offset of 1 starts the next cell
        self.Q[0:3][up] = 0.0
        self.C[up] += 1.0

    @property
    def n(self) -> int:
        return self.Q.shape[1]

    @property
    def P(self) -> np.ndarray:
        out = self.Q.copy()
        out[0:3] = self.C + self.Q[0:3]
        return out

    def copy(self) -> "Species":
        s = Species.__new__(Species)
        s.q, s.m, s.C, s.Q = self.q, self.m, self.C.copy(), self.Q.copy()
        return s


def courant_dt(d, courant: float = 0.5) -> float:
    """Time step at ``courant`` times the 3D Yee CFL limit, section 2.3, Eq. (15)."""
    d = np.asarray(d, dtype=np.float64)
    return courant / np.sqrt(np.sum(1.0 / d ** 2))


def faraday(n, d, dt, E, B, frac=1.0):
    """B <- B - frac*dt*curl E (section 2.3, Eq. (13)); E, B are (3, nz, ny, nx)."""
    n, d, pn, pd = _grid(n, d)
    lib().or_faraday(pn, pd, dt, _p(E), _p(B), frac)


def ampere(n, d, dt, E, B, J):
    """E <- E + dt (curl B - J) (section 2.3, Eq. (14))."""
    n, d, pn, pd = _grid(n, d)
    lib().or_ampere(pn, pd, dt, _p(E), _p(B), _p(J))


def gather(n, d, E, B, X, shape=1):
    """Staggered interpolation of E and B at one position X (cell units), section 2.5:
    CIC (shape 1) or the quadratic TSC weights (shape 2)."""
    n, d, pn, pd = _grid(n, d)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Ep = np.zeros(3)
    Bp = np.zeros(3)
    fn = lib().or_gather_tsc if shape == 2 else lib().or_gather
    fn(pn, pd, _p(np.ascontiguousarray(E)), _p(np.ascontiguousarray(B)), _p(X), _p(Ep), _p(Bp))
    return Ep, Bp


def boris(eps, E, B, u):
    """One relativistic Boris momentum update with eps = q dt / (2 m), section 2.4."""
    u = np.array(u, dtype=np.float64)
    lib().or_boris(eps, _p(np.ascontiguousarray(E, dtype=np.float64)),
                   _p(np.ascontiguousarray(B, dtype=np.float64)), _p(u))
    return u


def boris_orbit(E, B, qm, dt, x0, u0, nsteps, backpush=False):
    """Single particle in uniform E and B (section 3.1 problems): returns xs, us of
    shape (nsteps+1, 3); us[k] is u^{k-1/2}."""
    xs = np.zeros((nsteps + 1, 3))
    us = np.zeros((nsteps + 1, 3))
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().or_boris_orbit(_p(f(E)), _p(f(B)), qm, dt, _p(f(x0)), _p(f(u0)), nsteps, int(backpush), _p(xs), _p(us))
    return xs, us


def zigzag(n, d, dt, qw, X1, X2, J):
    """Accumulate the zigzag current of one move X1 -> X2 (cell units, X2 unwrapped) into J."""
    n, d, pn, pd = _grid(n, d)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().or_zigzag(pn, pd, dt, qw, _p(f(X1)), _p(f(X2)), _p(J))


def esirkepov(n, d, dt, qw, X1, X2, J):
    """Accumulate Esirkepov's current of one straight move X1 -> X2 (cell units, X2
    unwrapped, under one cell per dimension) into J, with the CIC shape."""
    n, d, pn, pd = _grid(n, d)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().or_esirkepov(pn, pd, dt, qw, _p(f(X1)), _p(f(X2)), _p(J))


def esirkepov_tsc(n, d, dt, qw, X1, X2, J):
    """Accumulate Esirkepov's current of one straight move X1 -> X2 (cell units, X2
    unwrapped, under one cell per dimension) into J, with the quadratic (TSC) shape."""
    n, d, pn, pd = _grid(n, d)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().or_esirkepov_tsc(pn, pd, dt, qw, _p(f(X1)), _p(f(X2)), _p(J))


def push(n, d, dt, E, Bn, species, J, esirkepov=False, shape=1):
    """The particle part of one cycle for one species (gather of E^n and B^n = ``Bn``,
    Boris, move, deposit into J), in place; returns the species' kinetic energy at the
    cycle's time level.  The same code as inside ``run``."""
    n_, d_, pn, pd = _grid(n, d)
    return lib().or_push(pn, pd, dt, _p(np.ascontiguousarray(E)), _p(np.ascontiguousarray(Bn)), species.q, species.m,
                         species.n, _p(species.Q), _p(species.C), _p(J), int(bool(esirkepov)), int(shape))


def rho(n, d, species, rho_ion=0.0, shape=1):
    """Node charge density: CIC (shape 1) or TSC (shape 2) of every species plus the
    uniform background rho_ion."""
    n, d, pn, pd = _grid(n, d)
    out = np.full(field_shape(n), float(rho_ion))
    fn = lib().or_rho_tsc if shape == 2 else lib().or_rho
    for s in species:
        fn(pn, pd, s.q, s.n, _p(s.Q), _p(s.C), _p(out))
    return out


def divergence(n, d, F):
    """Node divergence of an edge-located vector field (3, nz, ny, nx)."""
    n, d, pn, pd = _grid(n, d)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(F.shape[1:])
    lib().or_divergence(pn, pd, _p(F), _p(out))
    return out


def divergence_b(n, d, B):
    """Cell-centre divergence of a face-located field (3, nz, ny, nx)."""
    n, d, pn, pd = _grid(n, d)
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.zeros(B.shape[1:])
    lib().or_divergence_b(pn, pd, _p(B), _p(out))
    return out


def backpush(n, d, dt, E, Bhalf, species, shape=1):
    """u^0 -> u^{-1/2} by a backward Boris half step with E^0, B^0 (in place), the
    fields gathered with the CIC (shape 1) or TSC (shape 2) weights."""
    n, d, pn, pd = _grid(n, d)
    lib().or_backpush(pn, pd, dt, _p(np.ascontiguousarray(E)), _p(np.ascontiguousarray(Bhalf)),
                      species.q, species.m, species.n, _p(species.Q), _p(species.C), int(shape))


def run(n, d, dt, F, species, nsteps=1, step0=0, laser=None, current_filter=None, guide=None):
    """Advance the state ``F`` (9, nz, ny, nx[+1]) and the species in place by ``nsteps``
    cycles of Fig. 2.  Returns the (nsteps, 3) energy history (U_E, U_B, K) of the
    time levels n = 0 .. nsteps-1; on return F[6:9] holds the last J^{n+1/2}.
    ``step0`` is the index of the first cycle (it sets the laser time); ``laser`` =
    (a0, omega, w0, tau_fwhm, t_peak, i_s, yc, zc) adds the soft laser sheet;
    ``current_filter`` = (passes, compensate) filters the particle current each cycle
    (see ``current_filter``); ``guide`` = dict(pec_y, pec_z, port, e0, omega, tau,
    mode_y, esirkepov, shape) adds perfectly conducting walls on the planes y = 0 / z = 0,
    a hard TE port on the face x = 0 of an open x, with esirkepov = 1 deposits J with
    Esirkepov's scheme instead of ZigZag, and with shape = 2 uses the quadratic (TSC)
    particle shape for the gather and Esirkepov's deposit (see ``pic_oracle.c``)."""
    n, d, pn, pd = _grid(n, d)
    assert F.dtype == np.float64 and F.flags.c_contiguous and F.shape[0] == 9
    ns = len(species)
    qm = np.array([v for s in species for v in (s.q, s.m)], dtype=np.float64)
    npc = np.array([s.n for s in species], dtype=np.int64)
    ptrs = (_dp * ns)(*[_p(s.Q) for s in species])
    cptrs = (_dp * ns)(*[_p(s.C) for s in species])
    diag = np.zeros((nsteps, 3))
    las = None if laser is None else np.ascontiguousarray(laser, dtype=np.float64)
    filt = None if current_filter is None else np.ascontiguousarray(current_filter, dtype=np.float64)
    gd = None
    if guide is not None:
        gd = np.array([guide.get("pec_y", 0), guide.get("pec_z", 0), guide.get("port", 0), guide.get("e0", 0.0),
                       guide.get("omega", 0.0), guide.get("tau", 1.0), guide.get("mode_y", 1),
                       guide.get("esirkepov", 0), guide.get("shape", 1)], dtype=np.float64)
    lib().or_run(pn, pd, dt, _p(F), ns, _p(qm), npc.ctypes.data_as(_lp), ptrs, cptrs, nsteps, _p(diag), int(step0),
                 None if las is None else _p(las), None if filt is None else _p(filt),
                 None if gd is None else _p(gd))
    return diag


def current_filter(n, d, J, passes, compensate=True):
    """Filter J (3, nz, ny, nx[+1]) in place: along each dimension one convolution with
    `passes` binomial stencils (1/4, 1/2, 1/4) and, when compensating, the stencil
    (-p/4, 1 + p/2, -p/4); periodic dimensions wrap, an open x filters x = 0 .. nx-1
    with zero outside (the compensated binomial smoothing of section 2.2; reading, the
    paper gives no scheme)."""
    n_, d_, pn, pd = _grid(n, d)
    assert J.dtype == np.float64 and J.flags.c_contiguous
    lib().or_current_filter(pn, pd, _p(J), int(passes), int(bool(compensate)))


# --------------------------------------------------------------------------
# Moving window (section 2.2, the operations at the end of a cycle; section 4, the
# laser-wakefield run).  ``window`` is a dict:
#   start, every  the window moves one cell along +x after every cycle s with
#                 s >= start and (s - start) % every == every - 1;
#   species       index of the species that receives the new plasma;
#   ppc           (px, py, pz): the new plasma of a cell is a px x py x pz lattice at
#                 offsets (2a + 1) / (2 p) along each dimension, at rest;
#   density, x0, ramp   its density at absolute x (cell units): density * clip((x -
#                 x0) / ramp, 0, 1) (a step at x0 when ramp = 0); a particle carries
#                 weight density(x) dV / (px py pz), and none is made where it is 0.
# ``origin`` is the absolute x (cells) of the window's cell 0: the number of moves.

def window_moves_before(window, step):
    """Moves made by the cycles before ``step``."""
    s0, e = int(window["start"]), int(window["every"])
    return max(0, (int(step) - s0) // e) if step > s0 else 0


def window_moves_after(window, step):
    """Whether cycle ``step`` ends with a move."""
    s0, e = int(window["start"]), int(window["every"])
    return step >= s0 and (step - s0) % e == e - 1


def window_shift(n, d, F, species):
    """One move of the window (open x only): E and B shift one cell toward -x with a
    vacuum last column, particle cells drop by one and cell 0 leaves (weight 0)."""
    n_, d_, pn, pd = _grid(n, d)
    ns = len(species)
    npc = np.array([s.n for s in species], dtype=np.int64)
    ptrs = (_dp * ns)(*[_p(s.Q) for s in species])
    cptrs = (_dp * ns)(*[_p(s.C) for s in species])
    lib().or_window_shift(pn, pd, _p(F), ns, npc.ctypes.data_as(_lp), ptrs, cptrs)


def window_plasma(n, d, window, origin):
    """The new plasma of the window's last column when its cell 0 is at absolute x =
    ``origin``: a (7, m) array (positions in window cell units, momenta 0, weights),
    ordered by z cell, y cell, z offset, y offset, x offset (x fastest)."""
    nx, ny, nz = int(n[0]), int(n[1]), int(n[2])
    px, py, pz = (int(v) for v in window["ppc"])
    offx = (2 * np.arange(px) + 1) / (2.0 * px)
    offy = (2 * np.arange(py) + 1) / (2.0 * py)
    offz = (2 * np.arange(pz) + 1) / (2.0 * pz)
    X = float(origin + nx - 1) + offx                    # absolute x of the x offsets
    ramp = float(window["ramp"])
    if ramp > 0:
        prof = float(window["density"]) * np.clip((X - float(window["x0"])) / ramp, 0.0, 1.0)
    else:
        prof = float(window["density"]) * (X >= float(window["x0"]))
    w = prof * d[0] * d[1] * d[2] / (px * py * pz)
    a_on = np.nonzero(w > 0)[0]
    rows = []
    for k in range(nz):
        for j in range(ny):
            for c in range(pz):
                for b in range(py):
                    for a in a_on:
                        rows.append((nx - 1 + offx[a], j + offy[b], k + offz[c], 0.0, 0.0, 0.0, w[a]))
    if not rows:
        return np.zeros((7, 0))
    return np.array(rows, dtype=np.float64).T


def run_window(n, d, dt, F, species, nsteps, window, step0=0, laser=None, current_filter=None, guide=None):
    """``run`` with the moving window: after each cycle that ends with a move, the
    window shifts and species ``window["species"]`` receives the new column's plasma
    (appended in the order of ``window_plasma``).  ``guide`` is passed to ``run`` (the
    deposit and shape options).  Returns the (nsteps, 3) energy history."""
    origin = window_moves_before(window, step0)
    diag = np.zeros((nsteps, 3))
    for s in range(step0, step0 + nsteps):
        diag[s - step0] = run(n, d, dt, F, species, 1, step0=s, laser=laser, current_filter=current_filter,
                              guide=guide)[0]
        if window_moves_after(window, s):
            window_shift(n, d, F, species)
            origin += 1
            new = window_plasma(n, d, window, origin)
            if new.shape[1]:
                sp = species[int(window["species"])]
                add = Species(sp.q, sp.m, new)
                sp.C = np.ascontiguousarray(np.concatenate([sp.C, add.C], axis=1))
                sp.Q = np.ascontiguousarray(np.concatenate([sp.Q, add.Q], axis=1))
    return diag


def gauss_x(n, d, rho_total):
    """Ex from Gauss's law for charge varying along x only; returns (E (3,...), worst line mean)."""
    n, d, pn, pd = _grid(n, d)
    rho_total = np.ascontiguousarray(rho_total, dtype=np.float64)
    E = np.zeros((3,) + rho_total.shape)
    worst = lib().or_gauss_x(pn, pd, _p(rho_total), _p(E))
    return E, worst


def continuity_residual(n, d, dt, rho0, rho1, J):
    """R = (rho^{n+1} - rho^n)/dt + div J^{n+1/2} at the nodes, Eq. (12) in discrete form."""
    return (rho1 - rho0) / dt + divergence(n, d, J)


def empty_fields(n):
    return np.zeros((9,) + field_shape(n), dtype=np.float64)


# --------------------------------------------------------------------------
# Closed forms used as pins and as inputs.

def yee_omega(kvec, d, dt):
    """Numerical frequency of a vacuum plane wave on the Yee grid:
    (sin(w dt/2)/dt)^2 = sum_d (sin(k_d d_d/2)/d_d)^2  (the Yee dispersion relation)."""
    kvec = np.asarray(kvec, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    s = np.sqrt(np.sum((np.sin(kvec * d / 2) / d) ** 2))
    return 2.0 / dt * np.arcsin(s * dt)


def plane_wave(n, d, dt, mode, e_hat, amplitude, t_e=0.0):
    """Exact discrete vacuum eigenmode of the Yee scheme.

    ``mode`` = integer wave numbers (m_x, m_y, m_z) so that k_d = 2 pi m_d / (n_d d_d);
    ``e_hat`` = real polarisation vector, must be orthogonal to the discrete wave
    vector kappa_d = (2/d_d) sin(k_d d_d / 2).  Returns E (3,...) at time t_e and
    B (3,...) at time t_e - dt/2, each component sampled at its own Yee location,
    E = A e_hat sin(k.x - w t), B = A (kappa x e_hat)/Omega sin(k.x - w t), with
    Omega = (2/dt) sin(w dt/2) and w from ``yee_omega``."""
    n = [int(v) for v in n]
    d = np.asarray(d, dtype=np.float64)
    k = 2 * np.pi * np.asarray(mode, dtype=np.float64) / (np.asarray(n) * d)
    w = yee_omega(k, d, dt)
    kappa = 2.0 / d * np.sin(k * d / 2)
    e_hat = np.asarray(e_hat, dtype=np.float64)
    if abs(np.dot(kappa, e_hat)) > 1e-12 * np.linalg.norm(kappa) * np.linalg.norm(e_hat):
        raise ValueError("polarisation must be orthogonal to the discrete wave vector")
    Omega = 2.0 / dt * np.sin(w * dt / 2)
    b_hat = np.cross(kappa, e_hat) / Omega
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros((3, n[2], n[1], n[0]))
    half_e = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    half_b = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    for c in range(3):
        he = half_e[c]
        phase = k[0] * (ii + he[0]) * d[0] + k[1] * (jj + he[1]) * d[1] + k[2] * (kk + he[2]) * d[2]
        E[c] = amplitude * e_hat[c] * np.sin(phase - w * t_e)
        hb = half_b[c]
        phase = k[0] * (ii + hb[0]) * d[0] + k[1] * (jj + hb[1]) * d[1] + k[2] * (kk + hb[2]) * d[2]
        B[c] = amplitude * b_hat[c] * np.sin(phase - w * (t_e - dt / 2))
    return E, B, w


def cold_plasma_omega(k_cell, dt, omega_p=1.0):
    """Linear frequency of a cold-plasma Langmuir mode (wave number k_cell per cell)
    for sheets at cell offsets 1/4 and 3/4, with CIC charge on the nodes, Gauss's
    law on the edges and staggered linear gather, advanced by leapfrog:
    w_eff^2 = w_p^2 (1 - sin^2(k/2)/2), then sin(w dt/2) = w_eff dt/2.
    (Derivation: a sheet pair in cell m sets E(m+1/2) only; the gather weights
    1/4, 3/4 of the two sheets give the eigenvalue (3 + cos k)/4.)"""
    w_eff = omega_p * np.sqrt(1.0 - 0.5 * np.sin(k_cell / 2) ** 2)
    return 2.0 / dt * np.arcsin(w_eff * dt / 2)
