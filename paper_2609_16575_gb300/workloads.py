"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws and lays out numbers: particle positions (in cell units),
momenta and weights, grid sizes and the time step.  It holds none of the PIC
method's arithmetic, imports neither the CUDA binding nor the oracle, and is
the one piece both sides share.

Units are the paper's normalised units (c = eps0 = mu0 = 1, lengths in c/w_p,
times in 1/w_p); electrons have q = -1, m = 1; a uniform density n = 1 with
weight w = n dV / ppc gives w_p = 1.  Randomness comes from numpy's PCG64 with
a fixed seed per workload, so every run sees identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SpeciesInput:
    q: float
    m: float
    P: np.ndarray                      # (7, np) float64: X, Y, Z (cell units), ux, uy, uz, w
    momenta_at_half_step: bool = True  # False: P holds u^0 and the solver back-pushes to u^{-1/2}

    @property
    def n(self) -> int:
        return int(self.P.shape[1])


@dataclass
class Workload:
    name: str
    n: tuple                           # cells (nx, ny, nz)
    d: tuple                           # cell sizes
    dt: float
    rho_ion: float
    species: list = field(default_factory=list)
    E: np.ndarray | None = None        # optional initial E (3, nz, ny, nx); None = zero
    B: np.ndarray | None = None        # optional initial B^{-1/2}; None = zero
    steps: int = 1
    bc_x: int = 0                      # 1: open x (absorbing faces, particles leaving in x removed)
    laser: object = None               # LaserInput for an open x
    window: object = None              # WindowInput (moving window) for an open x

    @property
    def ncells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nparticles(self) -> int:
        return sum(s.n for s in self.species)


def courant_dt(d, courant=0.5) -> float:
    """Time step = courant x the 3D CFL limit 1/sqrt(sum 1/d^2)."""
    d = np.asarray(d, dtype=np.float64)
    return float(courant / np.sqrt(np.sum(1.0 / d ** 2)))


def _lattice(n, per_dim):
    """Regular lattice: per_dim^3 particles per cell at offsets (2a+1)/(2 per_dim)."""
    off = (2 * np.arange(per_dim) + 1) / (2.0 * per_dim)
    axes = [np.add.outer(np.arange(n[dd]), off).ravel() for dd in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def cold_plasma(n=16, d=0.1, per_dim=2, amplitude_cells=0.01, courant=0.5, steps=200) -> Workload:
    """Cold-plasma oscillation: periodic n^3 grid, per_dim^3 electrons per cell on a
    regular lattice, x-displacement amplitude_cells * dx * sin(2 pi x / L), zero momenta
    (given at t = 0), immobile neutralising ions.  The initial Ex that balances the
    displaced charge is left to the caller (it is a Gauss's-law solve)."""
    nn = (n, n, n)
    dd = (d, d, d)
    X, Y, Z = _lattice(nn, per_dim)
    X = X + amplitude_cells * np.sin(2 * np.pi * X / n)
    npart = X.size
    ppc = per_dim ** 3
    w = np.full(npart, d ** 3 / ppc)
    P = np.stack([X, Y, Z, np.zeros(npart), np.zeros(npart), np.zeros(npart), w])
    return Workload("cold_plasma", nn, dd, courant_dt(dd, courant), 1.0,
                    [SpeciesInput(-1.0, 1.0, P, momenta_at_half_step=False)], steps=steps)


def paper_cold_plasma(per_dim=2, v_amp=1e-3, courant=0.5, steps=2000) -> Workload:
    """The paper's plasma-oscillation setup (section 3.3): L = 2 pi per side, 2 x 2 x 100
    periodic cells, v_z = v_amp sin(z), quiet lattice start, immobile ions."""
    nn = (2, 2, 100)
    L = 2 * np.pi
    dd = (L / nn[0], L / nn[1], L / nn[2])
    X, Y, Z = _lattice(nn, per_dim)
    npart = X.size
    vz = v_amp * np.sin(Z * dd[2])
    uz = vz / np.sqrt(1 - vz ** 2)
    ppc = per_dim ** 3
    w = np.full(npart, dd[0] * dd[1] * dd[2] / ppc)
    P = np.stack([X, Y, Z, np.zeros(npart), np.zeros(npart), uz, w])
    return Workload("paper_cold_plasma", nn, dd, courant_dt(dd, courant), 1.0,
                    [SpeciesInput(-1.0, 1.0, P, momenta_at_half_step=False)], steps=steps)


def thermal(n=(128, 128, 128), d=0.2, ppc=64, u_th=0.05, seed=1235, courant=0.5, steps=100) -> Workload:
    """Thermal plasma: uniform random positions, Maxwellian momenta u_d ~ N(0, u_th^2)
    per component (given at the half step), immobile neutralising ions."""
    nn = tuple(int(v) for v in n)
    dd = (d, d, d)
    rng = np.random.Generator(np.random.PCG64(seed))
    ncell = nn[0] * nn[1] * nn[2]
    npart = ncell * ppc
    P = np.empty((7, npart))
    for dim in range(3):
        P[dim] = rng.random(npart) * nn[dim]
        # a draw of exactly n_d cannot happen (random() < 1), but rounding of the
        # product can; fold it back onto the periodic box
        P[dim][P[dim] >= nn[dim]] = 0.0
    for dim in range(3):
        P[3 + dim] = rng.standard_normal(npart) * u_th
    P[6] = d ** 3 / ppc
    return Workload("thermal", nn, dd, courant_dt(dd, courant), 1.0,
                    [SpeciesInput(-1.0, 1.0, P, momenta_at_half_step=True)], steps=steps)


def differentiable(n=32, d=0.2, ppc=16, u_th=0.02, seed=1237, courant=0.5, steps=200) -> Workload:
    """Particles of the differentiable run (32^3, 16 per cell, u_th = 0.02); the
    plane-wave field is added by the caller."""
    wl = thermal((n, n, n), d, ppc, u_th, seed, courant, steps)
    wl.name = "differentiable"
    return wl


def stress(n=256, d=0.2, ppc=32, u_th=0.1, seed=1238, courant=0.5, steps=1000) -> Workload:
    """Precision-stress thermal plasma: 256^3, 32 per cell, u_th = 0.1."""
    wl = thermal((n, n, n), d, ppc, u_th, seed, courant, steps)
    wl.name = "stress"
    return wl


@dataclass
class LaserInput:
    a0: float
    omega: float
    w0: float
    tau: float        # intensity FWHM
    t_peak: float
    plane: int
    yc: float         # cell units
    zc: float

    def as_tuple(self):
        return (self.a0, self.omega, self.w0, self.tau, self.t_peak, self.plane, self.yc, self.zc)


@dataclass
class WindowInput:
    """Moving window of an open x (see pic_window_desc): moves one cell along +x after
    every `every`-th cycle from `start`; the new column gets a ppc lattice of the density
    profile density * clip((X - x0) / ramp, 0, 1) at rest."""
    start: int
    every: int
    species: int
    ppc: tuple
    density: float
    x0: float
    ramp: float

    def as_tuple(self):
        return (self.start, self.every, self.species, self.ppc, self.density, self.x0, self.ramp)

    def as_dict(self):
        return dict(start=self.start, every=self.every, species=self.species, ppc=self.ppc, density=self.density,
                    x0=self.x0, ramp=self.ramp)


def lwfa(n=(512, 128, 128), ppc_per_dim=2, density=0.01, x0=20, ramp=50, a0=2.0, w0_lambda=8.0, fwhm_periods=10.0,
         courant=0.5, steps=2000, plane=2, window_start=None) -> Workload:
    """Laser wakefield in an underdense plasma (units of the laser: omega0 = 1, c = 1,
    lambda = 2 pi, density in units of the critical density): dx = lambda/20,
    dy = dz = lambda/8; open x (absorbing faces), periodic y and z; electrons on a
    regular per_dim^3 lattice where the density is non-zero: zero for x < x0 cells, a
    linear ramp over `ramp` cells, then `density`; zero momenta; immobile ions.  The
    linearly polarised (y) Gaussian pulse (a0, waist w0_lambda wavelengths, intensity
    FWHM fwhm_periods periods) enters through a current sheet on the node plane
    `plane`, peaking two FWHM after t = 0.  Returns the workload (bc_x = 1) with
    `.laser` set, and with `.window` set when window_start is given: a window moving one
    cell every ceil(dx / (c dt)) cycles from that cycle on (at or behind the speed of
    light) that brings in the same lattice and density profile."""
    lam = 2 * np.pi
    dd = (lam / 20, lam / 8, lam / 8)
    nn = tuple(int(v) for v in n)
    X, Y, Z = _lattice(nn, ppc_per_dim)
    prof = np.clip((X - x0) / ramp, 0.0, 1.0) * density
    keep = prof > 0
    X, Y, Z, prof = X[keep], Y[keep], Z[keep], prof[keep]
    ppc = ppc_per_dim ** 3
    w = prof * dd[0] * dd[1] * dd[2] / ppc
    npart = X.size
    P = np.stack([X, Y, Z, np.zeros(npart), np.zeros(npart), np.zeros(npart), w])
    wl = Workload("lwfa", nn, dd, courant_dt(dd, courant), 0.0,
                  [SpeciesInput(-1.0, 1.0, P, momenta_at_half_step=True)], steps=steps)
    tau = fwhm_periods * lam
    wl.laser = LaserInput(a0, 1.0, w0_lambda * lam, tau, 2.0 * tau, plane, nn[1] / 2.0, nn[2] / 2.0)
    wl.bc_x = 1
    if window_start is not None:
        every = int(np.ceil(dd[0] / wl.dt))
        wl.window = WindowInput(int(window_start), every, 0, (ppc_per_dim,) * 3, float(density), float(x0), float(ramp))
    return wl


def quantize_fp32(P: np.ndarray) -> np.ndarray:
    """Round a species array to what an FP32 cell + offset store can hold: the cell
    index stays exact, the in-cell offset, momenta and weight become float32 values.
    An offset that rounds up to 1.0 moves to offset 0 of the next cell."""
    Q = np.empty_like(P)
    for dim in range(3):
        c = np.floor(P[dim])
        off = (P[dim] - c).astype(np.float32).astype(np.float64)
        up = off >= 1.0
        c = c + up
        off[up] = 0.0
        Q[dim] = c + off
    Q[3:7] = P[3:7].astype(np.float32).astype(np.float64)
    return Q


def wrap_positions(P: np.ndarray, n) -> np.ndarray:
    """Fold positions onto the periodic box [0, n_d)."""
    Q = P.copy()
    for dim in range(3):
        Q[dim] = np.mod(Q[dim], n[dim])
        Q[dim][Q[dim] >= n[dim]] = 0.0
    return Q


def thermal_device(torch, n, d=0.2, ppc=32, u_th=0.1, seed=1238, courant=0.5, device="cuda"):
    """The thermal plasma drawn on the device with torch's Philox generator (for
    workloads too large to draw and upload from the host in reasonable time): positions
    uniform in [0, n_d) per dimension, then momenta N(0, u_th^2) per component (at the
    half step), weights d^3 / ppc.  Returns (X (3, N), U (3, N), w (N,), dt) as float64
    tensors on `device`; the same seed gives the same numbers on the same device type."""
    nn = tuple(int(v) for v in (n if hasattr(n, "__len__") else (n, n, n)))
    npart = nn[0] * nn[1] * nn[2] * int(ppc)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    X = torch.rand((3, npart), generator=gen, device=device, dtype=torch.float64)
    for dim in range(3):
        X[dim].mul_(nn[dim])
        # rounding of the product can give exactly n_d: fold it back into the box
        X[dim].masked_fill_(X[dim] >= nn[dim], 0.0)
    U = torch.randn((3, npart), generator=gen, device=device, dtype=torch.float64).mul_(u_th)
    w = torch.full((npart,), d ** 3 / ppc, device=device, dtype=torch.float64)
    return X, U, w, courant_dt((d, d, d), courant)
