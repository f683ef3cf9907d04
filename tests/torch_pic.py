"""A plain FP64 PyTorch (CPU, autograd) restatement of the PIC cycle of KEMPIC-3D
section 2.2, used only as an independent gradient reference on tiny grids.

Same discrete map as the oracle (Yee Eqs. (13)-(14), staggered CIC gather, Boris,
cell-relative move, zigzag deposit with the straight-segment flux term), written
with tensor operations so that autograd differentiates it.  Integer decisions
(cells, relay branches) are taken on detached values; the result is differentiable
wherever no particle changes a cell-crossing decision.
"""
from __future__ import annotations

import torch

HALF_E = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
HALF_B = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]


def curl_e(E, d):
    """C_E E at the B locations (Faraday, Eq. (13)); arrays are (3, nz, ny, nx)."""
    Ex, Ey, Ez = E
    nxt = lambda F, ax: torch.roll(F, -1, dims=ax)
    cx = (nxt(Ez, 1) - Ez) / d[1] - (nxt(Ey, 0) - Ey) / d[2]
    cy = (nxt(Ex, 0) - Ex) / d[2] - (nxt(Ez, 2) - Ez) / d[0]
    cz = (nxt(Ey, 2) - Ey) / d[0] - (nxt(Ex, 1) - Ex) / d[1]
    return torch.stack([cx, cy, cz])


def curl_b(B, d):
    """C_B B at the E locations (Ampere, Eq. (14))."""
    Bx, By, Bz = B
    prv = lambda F, ax: torch.roll(F, 1, dims=ax)
    cx = (Bz - prv(Bz, 1)) / d[1] - (By - prv(By, 0)) / d[2]
    cy = (Bx - prv(Bx, 0)) / d[2] - (Bz - prv(Bz, 2)) / d[0]
    cz = (By - prv(By, 2)) / d[0] - (Bx - prv(Bx, 1)) / d[1]
    return torch.stack([cx, cy, cz])


def _interp(F, C, x, half, n):
    """Trilinear interpolation of one staggered component at cells C + offsets x."""
    base, s = [], []
    for k in range(3):
        p = x[k] - 0.5 if half[k] else x[k]
        f = torch.floor(p.detach())
        base.append(C[k] + f.long())
        s.append(p - f)
    out = 0.0
    for c in range(2):
        for b in range(2):
            for a in range(2):
                wgt = (s[0] if a else 1 - s[0]) * (s[1] if b else 1 - s[1]) * (s[2] if c else 1 - s[2])
                idx = ((base[2] + c) % n[2], (base[1] + b) % n[1], (base[0] + a) % n[0])
                out = out + wgt * F[idx]
    return out


def _segment_add(J, cell, F, W, Cw, n):
    """Add one straight segment's 12 edge currents (zigzag with the D_p D_r / 12 term)."""
    N = n[0] * n[1] * n[2]
    flat = J.reshape(3, N)
    wx1, wy1, wz1 = W
    wx0, wy0, wz0 = 1 - wx1, 1 - wy1, 1 - wz1
    Fx, Fy, Fz = F
    t = 1.0 / 12.0
    entries = []
    for q in range(4):
        b, c = q & 1, q >> 1
        sg = 1.0 if b == c else -1.0
        entries.append((0, (0, b, c), Cw[0] * Fx * ((wy1 if b else wy0) * (wz1 if c else wz0) + sg * Fy * Fz * t)))
        entries.append((1, (b, 0, c), Cw[1] * Fy * ((wx1 if b else wx0) * (wz1 if c else wz0) + sg * Fx * Fz * t)))
        entries.append((2, (b, c, 0), Cw[2] * Fz * ((wx1 if b else wx0) * (wy1 if c else wy0) + sg * Fx * Fy * t)))
    rows = []
    for comp, (ox, oy, oz), val in entries:
        ix = (cell[0] + ox) % n[0]
        iy = (cell[1] + oy) % n[1]
        iz = (cell[2] + oz) % n[2]
        lin = (iz * n[1] + iy) * n[0] + ix
        rows.append(torch.zeros(3, N, dtype=J.dtype).index_put((torch.full_like(lin, comp), lin), val, accumulate=True))
    return (flat + sum(rows)).reshape(J.shape)


def step(E, B, C, x, u, w, q, m, n, d, dt):
    """One cycle.  State: E^n, B^{n-1/2} (3, nz, ny, nx); cells C (3, np) long; offsets x,
    momenta u (3, np); weights w (np).  Returns the next state and J^{n+1/2}."""
    h = 0.5 * dt
    Bn = B - h * curl_e(E, d)
    Ep = torch.stack([_interp(E[c], C, x, HALF_E[c], n) for c in range(3)])
    Bp = torch.stack([_interp(Bn[c], C, x, HALF_B[c], n) for c in range(3)])
    eps = q * dt / (2 * m)
    um = u + eps * Ep
    gm = torch.sqrt(1 + (um * um).sum(0))
    t = eps * Bp / gm
    s = 2 * t / (1 + (t * t).sum(0))
    up = um + torch.cross(um, t, dim=0)
    un = um + torch.cross(up, s, dim=0) + eps * Ep
    gn = torch.sqrt(1 + (un * un).sum(0))
    dtd = torch.tensor([dt / d[0], dt / d[1], dt / d[2]], dtype=x.dtype)[:, None]
    xe = x + dtd * un / gn
    st = torch.floor(xe.detach())
    x2 = xe - st
    tie = x2.detach() >= 1
    x2 = torch.where(tie, torch.zeros_like(x2), x2)
    st = (st + tie.to(st.dtype)).long()
    D = x2 - x
    F1 = torch.where(st == 0, 0.5 * D, torch.where(st > 0, 1 - x, -x))
    F2 = torch.where(st == 0, 0.5 * D, torch.where(st > 0, x2, x2 - 1))
    W1 = torch.where(st == 0, x + 0.25 * D, torch.where(st > 0, 0.5 * (x + 1), 0.5 * x))
    W2 = torch.where(st == 0, x + 0.75 * D, torch.where(st > 0, 0.5 * x2, 0.5 * (x2 + 1)))
    Cw = torch.stack([q * w / (dt * d[1] * d[2]), q * w / (dt * d[2] * d[0]), q * w / (dt * d[0] * d[1])])
    J = torch.zeros_like(E)
    J = _segment_add(J, C, F1, W1, Cw, n)
    J = _segment_add(J, C + st, F2, W2, Cw, n)
    Bh = Bn - h * curl_e(E, d)
    En = E + dt * (curl_b(Bh, d) - J)
    nt = torch.tensor(n, dtype=torch.long)[:, None]
    Cn = (C + st) % nt
    return En, Bh, Cn, x2, un, J


def field_energy(E, B, d, dt):
    """L = 1/2 dV sum (E^2 + B_N^2) with B_N = B^{N-1/2} - dt/2 curl E (Eq. (21))."""
    Bn = B - 0.5 * dt * curl_e(E, d)
    return 0.5 * d[0] * d[1] * d[2] * ((E * E).sum() + (Bn * Bn).sum())


def run(E, B, P, q, m, n, d, dt, nsteps):
    """P: (7, np) rows X, Y, Z (cell units), ux, uy, uz, w (tensors, may require grad)."""
    C = torch.floor(P[0:3].detach()).long()
    x = P[0:3] - C.to(P.dtype)
    u = P[3:6]
    w = P[6]
    for _ in range(nsteps):
        E, B, C, x, u, _ = step(E, B, C, x, u, w, q, m, n, d, dt)
    return E, B, C, x, u
