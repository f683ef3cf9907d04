"""``torch.autograd.Function`` over the library's checkpointed discrete adjoint.

``field_energy(u, amplitude, setup)`` returns the final field energy
L = U_E + U_B after ``setup["nsteps"]`` PIC cycles of one species with initial
momenta ``u`` (3, n) at t^{-1/2} and initial fields E^0 = A E_dir,
B^{-1/2} = A B_dir.  Its backward runs the hand-written adjoint kernels
(``pic_adjoint_backward``); this module only marshals arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gbpic


class FieldEnergyRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, amplitude, setup):
        s = setup
        pc = gbpic.Context(s["n"], s["d"], s["dt"], precision=s.get("precision", gbpic.PIC_FP64),
                           rho_ion=s.get("rho_ion", 0.0), track_ids=True, sort_every=s.get("sort_every", 0))
        A = float(amplitude)
        E_dir = np.ascontiguousarray(s["E_dir"], dtype=np.float64)
        B_dir = np.ascontiguousarray(s["B_dir"], dtype=np.float64)
        pc.set_fields(A * E_dir, A * B_dir)
        P = np.concatenate([np.asarray(s["X"], dtype=np.float64), u.detach().cpu().numpy().astype(np.float64),
                            np.asarray(s["w"], dtype=np.float64)[None, :]])
        pc.load_species_array(s["q"], s["m"], np.ascontiguousarray(P), momenta_at_half_step=True)
        L = pc.adjoint_forward(s["nsteps"], s.get("ckpt_every", 20))
        ctx.pc = pc
        ctx.dirs = (E_dir, B_dir)
        ctx.u_meta = (u.dtype, u.device)
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        dA, du = ctx.pc.adjoint_backward(*ctx.dirs)
        ctx.pc.close()
        dtype, device = ctx.u_meta
        g = float(gL)
        return (torch.from_numpy(du[0] * g).to(dtype=dtype, device=device),
                torch.tensor(dA * g, dtype=torch.float64), None)


def field_energy(u, amplitude, setup):
    return FieldEnergyRun.apply(u, amplitude, setup)
