"""Thin ctypes binding of the C ABI in ``include/gbpic.h``.

Argument marshalling only: every step of the PIC cycle runs in the CUDA kernels of
``libgbpic.so``.  The functions keep the C names (``pic_init_grid``, ``pic_step``,
...); ``Context`` wraps one ``pic_ctx`` for convenience.  PyTorch provides the
device memory (its caching allocator is passed to the library as the allocator)
and the stream; numpy arrays or CUDA torch tensors can be passed as inputs.

The library must have been built (``python -m paper_2609_16575_gb300.build`` or
``__graft_entry__.build()``); loading fails loudly when it is missing.  There is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbpic.so")

PIC_OK = 0
PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_OOM, PIC_ERR_CUDA, PIC_ERR_TILE_OVERFLOW = 1, 2, 3, 4, 5
PIC_ERR_SUPERLUMINAL, PIC_ERR_NAN, PIC_ERR_STATE, PIC_ERR_TIMEOUT, PIC_ERR_NO_DEVICE = 6, 7, 8, 9, 10
PIC_FP32 = 0
PIC_FP64 = 1
STATUS_NAMES = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_CFL", 3: "PIC_ERR_OOM", 4: "PIC_ERR_CUDA",
                5: "PIC_ERR_TILE_OVERFLOW", 6: "PIC_ERR_SUPERLUMINAL", 7: "PIC_ERR_NAN", 8: "PIC_ERR_STATE",
                9: "PIC_ERR_TIMEOUT", 10: "PIC_ERR_NO_DEVICE"}
PIC_DEPOSIT_ZIGZAG = 0
PIC_DEPOSIT_ESIRKEPOV = 1
PIC_SHAPE_CIC = 1
PIC_SHAPE_TSC = 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class pic_grid_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("d", ctypes.c_double * 3), ("dt", ctypes.c_double),
                ("rho_ion", ctypes.c_double), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("track_ids", ctypes.c_int32), ("record_every", ctypes.c_int32),
                ("history_capacity", ctypes.c_int32), ("sort_every", ctypes.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("bc_x", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class pic_laser_desc(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("omega", ctypes.c_double), ("w0", ctypes.c_double), ("tau", ctypes.c_double),
                ("t_peak", ctypes.c_double), ("plane", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("yc", ctypes.c_double), ("zc", ctypes.c_double)]


class pic_window_desc(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int32), ("every", ctypes.c_int32), ("species", ctypes.c_int32),
                ("ppc", ctypes.c_int32 * 3), ("density", ctypes.c_double), ("x0", ctypes.c_double),
                ("ramp", ctypes.c_double)]


class pic_port_desc(ctypes.Structure):
    _fields_ = [("e0", ctypes.c_double), ("omega", ctypes.c_double), ("tau", ctypes.c_double),
                ("mode_y", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pic_species_desc(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("n", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("u", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("momenta_at_half_step", ctypes.c_int32), ("device_pointers", ctypes.c_int32),
                ("capacity_slack", ctypes.c_double), ("mover_capacity", ctypes.c_int64),
                ("spill_capacity", ctypes.c_int64)]


class pic_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double), ("U_E", ctypes.c_double),
                ("U_B", ctypes.c_double), ("K_half", ctypes.c_double), ("gauss_max", ctypes.c_double),
                ("gauss_change_max", ctypes.c_double), ("rho_max", ctypes.c_double), ("cont_max", ctypes.c_double),
                ("J_max", ctypes.c_double), ("n_alive", ctypes.c_int64), ("n_spilled", ctypes.c_int64),
                ("n_escaped", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


class PicError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} {detail}".strip())


def lib():
    """Load libgbpic.so (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_16575_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.c_void_p
            L.pic_init_grid.argtypes = [ctypes.POINTER(pic_grid_desc), ctypes.POINTER(P)]
            L.pic_set_fields.argtypes = [P, P, P, ctypes.c_int32]
            L.pic_load_species.argtypes = [P, ctypes.POINTER(pic_species_desc), ctypes.POINTER(ctypes.c_int32)]
            L.pic_step.argtypes = [P, ctypes.c_int32]
            L.pic_sync.argtypes = [P]
            L.pic_get_fields.argtypes = [P, P, P, P, ctypes.c_int32]
            L.pic_get_particles.argtypes = [P, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
            L.pic_diagnostics.argtypes = [P, ctypes.POINTER(pic_diag)]
            L.pic_get_history.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
            L.pic_set_timing.argtypes = [P, ctypes.c_int32]
            L.pic_kernel_times.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_char_p),
                                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int32)]
            L.pic_adjoint_forward.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
            L.pic_adjoint_backward.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                               ctypes.c_int32]
            L.pic_set_laser.argtypes = [P, ctypes.POINTER(pic_laser_desc)]
            L.pic_set_moving_window.argtypes = [P, ctypes.POINTER(pic_window_desc)]
            L.pic_set_current_filter.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
            L.pic_set_pec.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
            L.pic_set_background.argtypes = [P, ctypes.c_double]
            L.pic_adjoint_run.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.c_int32]
            L.pic_set_deposit.argtypes = [P, ctypes.c_int32]
            L.pic_set_wait_limit.argtypes = [P, ctypes.c_int32]
            L.pic_set_shape.argtypes = [P, ctypes.c_int32]
            L.pic_set_shape.restype = ctypes.c_int
            L.pic_probe_fp64_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
            L.pic_save_state.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t)]
            L.pic_load_state.argtypes = [P, ctypes.c_void_p, ctypes.c_size_t]
            L.pic_free_state.argtypes = [ctypes.c_void_p]
            L.pic_free_state.restype = None
            L.pic_set_port.argtypes = [P, ctypes.POINTER(pic_port_desc)]
            L.pic_window_moves.argtypes = [P]
            L.pic_window_moves.restype = ctypes.c_int64
            L.pic_gauss_check_static.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.pic_launch_count.argtypes = [P]
            L.pic_launch_count.restype = ctypes.c_int64
            L.pic_last_error.argtypes = [P]
            L.pic_last_error.restype = ctypes.c_char_p
            L.pic_status_string.argtypes = [ctypes.c_int]
            L.pic_status_string.restype = ctypes.c_char_p
            L.pic_destroy.argtypes = [P]
            L.pic_destroy.restype = None
            for name in ("pic_init_grid", "pic_set_fields", "pic_load_species", "pic_step", "pic_sync",
                         "pic_get_fields", "pic_get_particles", "pic_diagnostics", "pic_get_history",
                         "pic_set_timing", "pic_kernel_times", "pic_adjoint_forward", "pic_adjoint_backward",
                         "pic_gauss_check_static", "pic_set_laser", "pic_set_moving_window",
                         "pic_set_current_filter", "pic_set_pec", "pic_set_port", "pic_set_deposit",
                         "pic_save_state", "pic_load_state", "pic_set_background", "pic_adjoint_run",
                         "pic_set_wait_limit", "pic_probe_fp64_rate"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


EXPORTED = ("pic_init_grid", "pic_set_fields", "pic_load_species", "pic_step", "pic_sync", "pic_get_fields",
            "pic_get_particles", "pic_diagnostics", "pic_get_history", "pic_set_timing", "pic_kernel_times",
            "pic_adjoint_forward", "pic_adjoint_backward", "pic_gauss_check_static", "pic_set_laser", "pic_launch_count",
            "pic_last_error", "pic_status_string", "pic_destroy")


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data, 0
    # torch tensor
    assert a.is_contiguous() and str(a.dtype) == "torch.float64"
    return a.data_ptr(), 1 if a.is_cuda else 0


def _check(ctx_ptr, status, what):
    if status != PIC_OK:
        detail = lib().pic_last_error(ctx_ptr).decode() if ctx_ptr else ""
        raise PicError(status, what, detail)


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device, stream):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None

        def _free(p, user):
            torch.cuda.caching_allocator_delete(p)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def pic_init_grid(n, d, dt, precision=PIC_FP32, rho_ion=0.0, device=0, stream=None, track_ids=False,
                  record_every=0, history_capacity=0, allocator=None, sort_every=0, bc_x=0):
    """Create a context; returns (ctx pointer, keep-alive tuple)."""
    desc = pic_grid_desc()
    desc.n = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    desc.d = (ctypes.c_double * 3)(*[float(v) for v in d])
    desc.dt = float(dt)
    desc.rho_ion = float(rho_ion)
    desc.precision = int(precision)
    desc.device = int(device)
    desc.stream = stream
    desc.track_ids = int(bool(track_ids))
    desc.record_every = int(record_every)
    desc.history_capacity = int(history_capacity)
    desc.sort_every = int(sort_every)
    desc.bc_x = int(bc_x)
    if allocator is not None:
        desc.alloc = allocator.alloc
        desc.free = allocator.free
    out = ctypes.c_void_p()
    _check(None, lib().pic_init_grid(ctypes.byref(desc), ctypes.byref(out)), "pic_init_grid")
    return out, (desc, allocator)


def probe_fp64_rate(device=0):
    """FP64 FMA rate of the device in FLOP/s (pic_probe_fp64_rate)."""
    v = ctypes.c_double()
    _check(None, lib().pic_probe_fp64_rate(int(device), ctypes.byref(v)), "pic_probe_fp64_rate")
    return v.value


class Context:
    """One pic_ctx.  ``use_torch`` routes allocations through torch's caching allocator
    and enqueues on torch's current stream of ``device``."""

    def __init__(self, n, d, dt, precision=PIC_FP32, rho_ion=0.0, device=0, track_ids=False, record_every=0,
                 history_capacity=0, use_torch=True, sort_every=0, bc_x=0, allocator=None):
        """``allocator``: an object with ``alloc``/``free`` callbacks (ALLOC_FN, FREE_FN) in
        place of torch's caching allocator (the stream stays torch's)."""
        stream = None
        if use_torch:
            import torch

            torch.cuda.init()
            s = torch.cuda.current_stream(device)
            # torch's default stream has handle 0; pass cudaStreamLegacy (0x1) so that the
            # library enqueues on that same stream instead of creating its own
            stream = s.cuda_stream or 1
            if allocator is None:
                allocator = _TorchAllocator(device, s.cuda_stream)
        self.n = tuple(int(v) for v in n[:3])
        self.bc_x = int(bc_x)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.ptr, self._keep = pic_init_grid(self.n, d, dt, precision, rho_ion, device, stream, track_ids,
                                             record_every, history_capacity, allocator, sort_every, bc_x)
        self.species_n = []

    def close(self):
        if self.ptr:
            lib().pic_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, E=None, B=None):
        """E^0, B^{-1/2}: (3, nz, ny, nx [+ 1 with an open x]) float64 each, or None."""
        want = 3 * self.n[2] * self.n[1] * (self.n[0] + self.bc_x)
        for a in (E, B):
            if a is not None and int(np.prod(a.shape)) != want:
                raise ValueError(f"field array of {int(np.prod(a.shape))} values, expected {want}")
        pe, de = _ptr(E)
        pb, db = _ptr(B)
        if E is not None and B is not None and de != db:
            raise ValueError("E and B must both be host or both be device arrays")
        _check(self.ptr, lib().pic_set_fields(self.ptr, pe, pb, de or db), "pic_set_fields")

    def load_species(self, q, m, X, u, w, momenta_at_half_step=True, capacity_slack=0.0, mover_capacity=0,
                     spill_capacity=0):
        """X, u: (3, n) float64; w: (n,) float64 (numpy or CUDA torch)."""
        n = int(w.shape[0])
        desc = pic_species_desc()
        desc.q, desc.m, desc.n = float(q), float(m), n
        px, dx = _ptr(X)
        pu, du = _ptr(u)
        pw, dw = _ptr(w)
        if not (dx == du == dw):
            raise ValueError("X, u, w must all be host or all be device arrays")
        desc.X, desc.u, desc.w = px, pu, pw
        desc.momenta_at_half_step = int(bool(momenta_at_half_step))
        desc.device_pointers = dx
        desc.capacity_slack = float(capacity_slack)
        desc.mover_capacity = int(mover_capacity)
        desc.spill_capacity = int(spill_capacity)
        sid = ctypes.c_int32()
        _check(self.ptr, lib().pic_load_species(self.ptr, ctypes.byref(desc), ctypes.byref(sid)), "pic_load_species")
        self.species_n.append(n)
        return sid.value

    def load_species_array(self, q, m, P, momenta_at_half_step=True, capacity_slack=0.0, mover_capacity=0,
                           spill_capacity=0):
        """P: (7, n) float64 rows X, Y, Z, ux, uy, uz, w."""
        if isinstance(P, np.ndarray):
            P = np.ascontiguousarray(P, dtype=np.float64)
            return self.load_species(q, m, np.ascontiguousarray(P[0:3]), np.ascontiguousarray(P[3:6]),
                                     np.ascontiguousarray(P[6]), momenta_at_half_step, capacity_slack, mover_capacity,
                                     spill_capacity)
        return self.load_species(q, m, P[0:3].contiguous(), P[3:6].contiguous(), P[6].contiguous(),
                                 momenta_at_half_step, capacity_slack, mover_capacity, spill_capacity)

    def step(self, nsteps=1):
        _check(self.ptr, lib().pic_step(self.ptr, int(nsteps)), "pic_step")

    def sync(self):
        _check(self.ptr, lib().pic_sync(self.ptr), "pic_sync")

    def get_fields(self):
        """Returns E, B, J as (3, nz, ny, nx) float64 numpy arrays (E^n, B^{n-1/2}, J^{n-1/2})."""
        shape = (3, self.n[2], self.n[1], self.n[0] + self.bc_x)
        E = np.empty(shape)
        B = np.empty(shape)
        J = np.empty(shape)
        _check(self.ptr, lib().pic_get_fields(self.ptr, E.ctypes.data, B.ctypes.data, J.ctypes.data, 0),
               "pic_get_fields")
        return E, B, J

    def get_particles(self, species=0):
        n = ctypes.c_int64()
        _check(self.ptr, lib().pic_get_particles(self.ptr, species, None, ctypes.byref(n), 0), "pic_get_particles")
        out = np.empty((7, n.value))
        _check(self.ptr, lib().pic_get_particles(self.ptr, species, out.ctypes.data, ctypes.byref(n), 0),
               "pic_get_particles")
        return out

    def diagnostics(self):
        d = pic_diag()
        _check(self.ptr, lib().pic_diagnostics(self.ptr, ctypes.byref(d)), "pic_diagnostics")
        return d.as_dict()

    def log_diagnostics(self, path, **extra):
        """Append the current diagnostics (and any extra keys) to a JSON-lines file; returns
        the record."""
        import json
        import time

        rec = dict(self.diagnostics(), wall_time=time.time(), **extra)
        with open(path, "a") as f:
            f.write(json.dumps({k: (v if not isinstance(v, float) or math.isfinite(v) else None)
                                for k, v in rec.items()}) + "\n")
        return rec

    def history(self, max_records=1 << 16):
        cnt = ctypes.c_int32()
        out = np.zeros((max_records, 3))
        _check(self.ptr, lib().pic_get_history(self.ptr, out.ctypes.data, max_records, ctypes.byref(cnt)),
               "pic_get_history")
        return out[:cnt.value]

    def set_wait_limit(self, polls):
        _check(self.ptr, lib().pic_set_wait_limit(self.ptr, int(polls)), "pic_set_wait_limit")

    def set_timing(self, enable=True):
        _check(self.ptr, lib().pic_set_timing(self.ptr, int(bool(enable))), "pic_set_timing")

    def kernel_times(self):
        """{kernel class: (launches, total ms)} accumulated since the last call."""
        k = 16
        names = (ctypes.c_char_p * k)()
        launches = (ctypes.c_int64 * k)()
        ms = (ctypes.c_double * k)()
        cnt = ctypes.c_int32()
        _check(self.ptr, lib().pic_kernel_times(self.ptr, k, names, launches, ms, ctypes.byref(cnt)),
               "pic_kernel_times")
        return {names[i].decode(): (launches[i], ms[i]) for i in range(cnt.value)}

    def launch_count(self):
        return lib().pic_launch_count(self.ptr)

    def set_laser(self, a0, omega, w0, tau, t_peak, plane, yc, zc):
        """Laser sheet of an open x (see pic_laser_desc)."""
        L = pic_laser_desc(a0, omega, w0, tau, t_peak, int(plane), 0, yc, zc)
        _check(self.ptr, lib().pic_set_laser(self.ptr, ctypes.byref(L)), "pic_set_laser")

    def set_moving_window(self, start, every, species, ppc, density, x0, ramp):
        """Moving window of an open x (see pic_window_desc); before loading `species`."""
        W = pic_window_desc(int(start), int(every), int(species), (ctypes.c_int32 * 3)(*[int(v) for v in ppc]),
                            float(density), float(x0), float(ramp))
        _check(self.ptr, lib().pic_set_moving_window(self.ptr, ctypes.byref(W)), "pic_set_moving_window")

    def set_current_filter(self, passes, compensate=True):
        """Compensated binomial current filter (see pic_set_current_filter); 0 passes: off."""
        _check(self.ptr, lib().pic_set_current_filter(self.ptr, int(passes), int(compensate)),
               "pic_set_current_filter")

    def save_state(self):
        """The dynamical state as bytes (see pic_save_state)."""
        blob, size = ctypes.c_void_p(), ctypes.c_size_t()
        _check(self.ptr, lib().pic_save_state(self.ptr, ctypes.byref(blob), ctypes.byref(size)), "pic_save_state")
        try:
            return ctypes.string_at(blob, size.value)
        finally:
            lib().pic_free_state(blob)

    def load_state(self, data):
        """Restore a state from save_state into this fresh context (see pic_load_state)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(self.ptr, lib().pic_load_state(self.ptr, buf, len(data)), "pic_load_state")

    def set_deposit(self, scheme):
        """PIC_DEPOSIT_ZIGZAG (0, default) or PIC_DEPOSIT_ESIRKEPOV (1)."""
        _check(self.ptr, lib().pic_set_deposit(self.ptr, int(scheme)), "pic_set_deposit")

    def set_shape(self, shape):
        """PIC_SHAPE_CIC (1, default) or PIC_SHAPE_TSC (2: quadratic shape, Esirkepov's deposit)."""
        _check(self.ptr, lib().pic_set_shape(self.ptr, int(shape)), "pic_set_shape")

    def set_background(self, rho_ion):
        """Uniform immobile background charge density (diagnostics only)."""
        _check(self.ptr, lib().pic_set_background(self.ptr, float(rho_ion)), "pic_set_background")

    def set_pec(self, pec_y, pec_z):
        """Conducting wall planes y = 0 / z = 0 (see pic_set_pec); fields only."""
        _check(self.ptr, lib().pic_set_pec(self.ptr, int(pec_y), int(pec_z)), "pic_set_pec")

    def set_port(self, e0, omega, tau, mode_y=1):
        """Hard TE port on the face x = 0 of an open x (see pic_port_desc)."""
        P = pic_port_desc(float(e0), float(omega), float(tau), int(mode_y), 0)
        _check(self.ptr, lib().pic_set_port(self.ptr, ctypes.byref(P)), "pic_set_port")

    def window_moves(self):
        """Moves of the window so far."""
        return int(lib().pic_window_moves(self.ptr))

    def gauss_check_static(self):
        """(gauss_max, rho_max) from the allocation-free entry point."""
        g, r = ctypes.c_double(), ctypes.c_double()
        _check(self.ptr, lib().pic_gauss_check_static(self.ptr, ctypes.byref(g), ctypes.byref(r)),
               "pic_gauss_check_static")
        return g.value, r.value

    def adjoint_forward(self, nsteps, ckpt_every):
        """Advance nsteps keeping checkpoints; returns L = U_E + U_B of the final state."""
        L = ctypes.c_double()
        _check(self.ptr, lib().pic_adjoint_forward(self.ptr, int(nsteps), int(ckpt_every), ctypes.byref(L)),
               "pic_adjoint_forward")
        return L.value

    def adjoint_backward(self, E_dir=None, B_dir=None):
        """Gradients of the last adjoint_forward loss: (dL/dA, [dL/du^{-1/2} (3, n) per species])."""
        outs = [np.zeros((3, n)) for n in self.species_n]
        ptrs = (ctypes.c_void_p * max(len(outs), 1))(*[o.ctypes.data for o in outs])
        dA = ctypes.c_double()
        pe, _ = _ptr(E_dir)
        pb, _ = _ptr(B_dir)
        _check(self.ptr, lib().pic_adjoint_backward(self.ptr, pe, pb, ctypes.byref(dA), ptrs, 0),
               "pic_adjoint_backward")
        return dA.value, outs

    def adjoint_run(self, nsteps, ckpt_every, E_dir=None, B_dir=None):
        """Forward and backward in one call: (loss, dL/dA, [dL/du^{-1/2} per species])."""
        outs = [np.zeros((3, n)) for n in self.species_n]
        ptrs = (ctypes.c_void_p * max(len(outs), 1))(*[o.ctypes.data for o in outs])
        loss, dA = ctypes.c_double(), ctypes.c_double()
        pe, _ = _ptr(E_dir)
        pb, _ = _ptr(B_dir)
        _check(self.ptr, lib().pic_adjoint_run(self.ptr, int(nsteps), int(ckpt_every), pe, pb, ctypes.byref(loss),
                                               ctypes.byref(dA), ptrs, 0), "pic_adjoint_run")
        return loss.value, dA.value, outs
