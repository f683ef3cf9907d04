"""Spatial domain decomposition of the PIC cycle along x, run with the FP64 oracle on CPU
ranks (test infrastructure: the library runs one GPU, and this shows how the cycle
shards and that the sharded cycle is the same computation).

Rank r of W owns the x-slab of cells [r w, (r + 1) w), w = n_x / W, of a periodic box.
It keeps the slab on a local periodic box of w + 2 H cells along x: H halo planes on
each side, which hold copies of the neighbours' edge planes.  One cycle (section 2.2,
Fig. 2) on a rank:
  1. halo exchange: E and B planes [H, 2H) go to the left neighbour's right halo,
     [w, w + H) to the right neighbour's left halo;
  2. B^{n+1/2} = B^{n-1/2} - dt curl E^n on the local box (exact on the slab and on the
     first halo plane), B^n the average;
  3. the slab's particles: gather, Boris, move and deposit into the local J (a particle
     moves less than a cell, so its current stays within one halo plane);
  4. current fold: J on the halo planes is added to the neighbours' edge planes;
  5. E^{n+1} = E^n + dt (curl B^{n+1/2} - J) on the local box (exact on the slab);
  6. migration: particles whose cell left the slab go to the neighbour that owns it.
The exchanges are point-to-point sends between neighbours (torch.distributed).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

import oracle

H = 2   # halo planes per side


def _exchange(sends, recvs):
    """Point-to-point exchange without deadlock: sends = [(array, peer, tag)], recvs =
    [(shape, peer, tag)]; returns the received arrays in the order of recvs."""
    reqs, outs = [], []
    for a, p, t in sends:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)), p, tag=t))
    for shp, p, t in recvs:
        buf = torch.zeros(shp, dtype=torch.float64)
        reqs.append(dist.irecv(buf, p, tag=t))
        outs.append(buf)
    for r in reqs:
        r.wait()
    return [o.numpy() for o in outs]


class Slab:
    """One rank's share of a periodic box: fields (9, nz, ny, w + 2H) and the particles
    of its slab (cells local: x + H - x0) with their load-order ids."""

    def __init__(self, n, d, dt, F, P, q, m, rank, world):
        assert n[0] % world == 0 and n[0] // world >= H
        self.n, self.d, self.dt = tuple(n), tuple(d), dt
        self.rank, self.world = rank, world
        self.w = n[0] // world
        self.x0 = rank * self.w
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.nl = (self.w + 2 * H, n[1], n[2])
        gx = (np.arange(self.w + 2 * H) - H + self.x0) % n[0]
        self.F = np.ascontiguousarray(F[..., gx])
        sp = oracle.Species(q, m, P)
        own = (sp.C[0] >= self.x0) & (sp.C[0] < self.x0 + self.w)
        self.sp = oracle.Species(q, m, np.zeros((7, 0)))
        self.sp.C = np.ascontiguousarray(sp.C[:, own])
        self.sp.C[0] += H - self.x0
        self.sp.Q = np.ascontiguousarray(sp.Q[:, own])
        self.ids = np.nonzero(own)[0].astype(np.float64)
        self.migrated = 0
        self.folded = 0.0

    def _exchange_halos(self, A):
        """A (c, nz, ny, w + 2H): fill both halos from the neighbours' edge planes."""
        w = self.w
        to_left, to_right = A[..., H:2 * H], A[..., w:w + H]
        # tag 0: a rank's first planes, sent leftwards; tag 1: its last planes, rightwards
        from_right, from_left = _exchange([(to_left, self.left, 0), (to_right, self.right, 1)],
                                          [(to_left.shape, self.right, 0), (to_right.shape, self.left, 1)])
        A[..., 0:H] = from_left
        A[..., w + H:w + 2 * H] = from_right

    def _fold_current(self, J):
        """Add the current deposited on the halo planes to the neighbours' edge planes."""
        w = self.w
        to_left, to_right = J[..., 0:H].copy(), J[..., w + H:w + 2 * H].copy()
        self.folded += np.abs(to_left).sum() + np.abs(to_right).sum()
        # tag 2: a rank's left-halo current, sent leftwards; tag 3: its right-halo current
        from_right, from_left = _exchange([(to_left, self.left, 2), (to_right, self.right, 3)],
                                          [(to_left.shape, self.right, 2), (to_right.shape, self.left, 3)])
        J[..., w:w + H] += from_right      # the right neighbour's left halo lies on my last planes
        J[..., H:2 * H] += from_left       # the left neighbour's right halo lies on my first planes
        J[..., 0:H] = 0.0
        J[..., w + H:w + 2 * H] = 0.0

    def _migrate(self):
        """Send the particles whose cell left the slab to the neighbour that owns it."""
        sp, w = self.sp, self.w
        cx = sp.C[0]
        go_l, go_r = cx < H, cx >= H + w
        stay = ~(go_l | go_r)
        packs = []
        for sel, shift in ((go_l, w), (go_r, -w)):
            C = sp.C[:, sel].copy()
            C[0] += shift          # the receiver's local cell
            pack = np.concatenate([C, sp.Q[:, sel], self.ids[sel][None, :]], axis=0)
            # one padding column, so that no message is empty
            packs.append(np.concatenate([pack, np.zeros((11, 1))], axis=1))
        self.migrated += int(go_l.sum() + go_r.sum())
        counts = np.array([float(packs[0].shape[1]), float(packs[1].shape[1])])
        # tag 4 / 6: the left-going count / pack; tag 5 / 7: the right-going ones
        c_right, c_left = _exchange([(counts, self.left, 4), (counts, self.right, 5)],
                                    [((2,), self.right, 4), ((2,), self.left, 5)])
        from_right, from_left = _exchange([(packs[0], self.left, 6), (packs[1], self.right, 7)],
                                          [((11, int(c_right[0])), self.right, 6), ((11, int(c_left[1])), self.left, 7)])
        from_right, from_left = from_right[:, :-1], from_left[:, :-1]
        sp.C = np.ascontiguousarray(np.concatenate([sp.C[:, stay], from_left[0:3], from_right[0:3]], axis=1))
        sp.Q = np.ascontiguousarray(np.concatenate([sp.Q[:, stay], from_left[3:10], from_right[3:10]], axis=1))
        self.ids = np.concatenate([self.ids[stay], from_left[10], from_right[10]])

    def step(self):
        F = self.F
        self._exchange_halos(F[0:6])
        E, B, J = F[0:3], F[3:6], F[6:9]
        Bold = B.copy()
        oracle.faraday(self.nl, self.d, self.dt, E, B, 1.0)
        Bn = 0.5 * (B + Bold)
        J[...] = 0.0
        oracle.push(self.nl, self.d, self.dt, E, Bn, self.sp, J)
        self._fold_current(J)
        oracle.ampere(self.nl, self.d, self.dt, E, B, J)
        self._migrate()

    def result(self):
        """The slab's fields (9, nz, ny, w) and its particles as (ids, 7 rows of global X,
        Y, Z, ux, uy, uz, w)."""
        F = self.F[..., H:H + self.w].copy()
        C = self.sp.C.copy()
        C[0] += self.x0 - H
        P = self.sp.Q.copy()
        P[0:3] = C + self.sp.Q[0:3]
        return F, self.ids.astype(np.int64), P
