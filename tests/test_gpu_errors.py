"""Failure detection on the device without faulting it: bad inputs that the kernels
detect set an error bit, the next synchronising call returns the status, and the
process can carry on with a fresh context."""
import numpy as np
import pytest

from paper_2609_16575_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(gbpic, wl, prec):
    return gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=wl.rho_ion, track_ids=True)


@pytest.mark.parametrize("prec", [0, 1])
def test_non_finite_momentum_is_reported(prec):
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=71)
    P = wl.species[0].P.copy()
    P[4, 17] = np.nan
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, P)
    with pytest.raises(gbpic.PicError) as e:
        ctx.step(2)
        ctx.sync()
    assert e.value.status == gbpic.PIC_ERR_NAN
    ctx.close()
    # a fresh context on the same device works
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    ctx.step(2)
    ctx.sync()
    assert ctx.diagnostics()["n_alive"] == wl.species[0].P.shape[1]
    ctx.close()


def test_positions_outside_the_box_are_rejected_at_load():
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=72)
    P = wl.species[0].P.copy()
    P[1, 3] = 8.0          # y = n_y is outside [0, n_y)
    ctx = _ctx(gbpic, wl, 0)
    with pytest.raises(gbpic.PicError) as e:
        ctx.load_species_array(-1.0, 1.0, P)
    assert e.value.status == gbpic.PIC_ERR_ARG
    P[1, 3] = 7.5
    P[6, 5] = -1.0         # weights must be positive
    with pytest.raises(gbpic.PicError) as e:
        ctx.load_species_array(-1.0, 1.0, P)
    assert e.value.status == gbpic.PIC_ERR_ARG
    ctx.close()


def test_adjoint_needs_ids_and_a_periodic_box():
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 8, 8), 0.2, 2, 0.05, seed=73)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=1, rho_ion=wl.rho_ion, track_ids=False)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError):
        ctx.adjoint_forward(4, 2)
    ctx.close()
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=1, rho_ion=0.0, track_ids=True, bc_x=1)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError):
        ctx.adjoint_forward(4, 2)
    ctx.close()


def test_adjoint_backward_refuses_a_changed_species_set():
    """The backward pass needs the species of its forward pass: without a forward pass,
    and after a species was loaded since, it returns PIC_ERR_STATE; a new forward pass
    (which reserves its memory again) makes it work."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((8, 8, 8), 0.2, 2, 0.05, seed=75)
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=1, rho_ion=0.0, track_ids=True)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError) as e:
        ctx.adjoint_backward()
    assert e.value.status == gbpic.PIC_ERR_STATE
    ctx.adjoint_forward(4, 2)
    ctx.load_species_array(1.0, 1836.0, wl.species[0].P)
    with pytest.raises(gbpic.PicError) as e:
        ctx.adjoint_backward()
    assert e.value.status == gbpic.PIC_ERR_STATE
    assert b"species changed" in gbpic.lib().pic_last_error(ctx.ptr)
    ctx.adjoint_forward(4, 2)
    _, du = ctx.adjoint_backward()
    assert len(du) == 2 and all(np.isfinite(g).all() for g in du)
    ctx.close()


# --- failures made on the host, reported by the library without faulting the device ---

@pytest.mark.parametrize("prec", [0, 1])
def test_staging_wait_timeout_is_reported(prec):
    """A staging wait bounded to zero polls gives up in every tile: the tile kernel raises
    its timeout bit (after its copies have landed) and pic_sync returns PIC_ERR_TIMEOUT;
    a fresh context on the same device then steps normally."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 16, 8), 0.2, 4, 0.1, seed=74)
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    ctx.set_wait_limit(0)
    ctx.step(1)
    with pytest.raises(gbpic.PicError) as e:
        ctx.sync()
    assert e.value.status == gbpic.PIC_ERR_TIMEOUT
    assert b"wait" in gbpic.lib().pic_last_error(ctx.ptr)
    ctx.close()
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    ctx.set_wait_limit(-1)          # the default bound
    ctx.step(2)
    ctx.sync()
    assert ctx.diagnostics()["n_alive"] == wl.species[0].P.shape[1]
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_mover_list_overflow_is_reported(prec):
    """A mover list shrunk on the host (64 records) against a hot plasma that sends
    hundreds of particles across tile faces per step: the step drops the excess and
    pic_sync returns PIC_ERR_TILE_OVERFLOW."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 16, 16), 0.2, 4, 0.3, seed=75)
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P, mover_capacity=64)
    ctx.step(1)
    with pytest.raises(gbpic.PicError) as e:
        ctx.sync()
    assert e.value.status == gbpic.PIC_ERR_TILE_OVERFLOW
    assert b"overflow" in gbpic.lib().pic_last_error(ctx.ptr)
    ctx.close()
    # the default capacities carry the same run
    ctx = _ctx(gbpic, wl, prec)
    ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    ctx.step(3)
    ctx.sync()
    assert ctx.diagnostics()["n_alive"] == wl.species[0].P.shape[1]
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_spill_list_overflow_is_reported(prec):
    """A beam of 2000 particles crossing into an empty tile (segment of 32 slots) in one
    step: the arrivals that do not fit go to the spill list, shrunk on the host to 64
    records, which overflows: PIC_ERR_TILE_OVERFLOW.  With the default spill list the
    same beam is carried without loss."""
    from paper_2609_16575_gb300 import gbpic

    n = (16, 8, 8)
    rng = np.random.default_rng(76)
    m = 2000
    P = np.zeros((7, m))
    P[0] = 7.8 + 0.19 * rng.random(m)     # the last x column of tile 0, moving +x at ~0.95 c
    P[1] = 8 * rng.random(m)
    P[2] = 8 * rng.random(m)
    P[3] = 3.0
    P[6] = 1e-3
    d = (0.2, 0.2, 0.2)
    dt = W.courant_dt(d, 0.5)
    for spill, ok in ((64, False), (0, True)):
        ctx = gbpic.Context(n, d, dt, precision=prec, track_ids=True)
        ctx.load_species_array(-1.0, 1.0, P, capacity_slack=1e-9, spill_capacity=spill)
        ctx.step(1)
        if ok:
            ctx.sync()
            diag = ctx.diagnostics()
            assert diag["n_alive"] == m and diag["n_spilled"] > 0
        else:
            with pytest.raises(gbpic.PicError) as e:
                ctx.sync()
            assert e.value.status == gbpic.PIC_ERR_TILE_OVERFLOW
        ctx.close()


class _BudgetAllocator:
    """Device allocations through torch's caching allocator up to a byte budget; past it
    the callback returns NULL, as an exhausted memory pool would."""

    def __init__(self, budget):
        import torch
        from paper_2609_16575_gb300 import gbpic

        self.used = 0
        self.budget = budget
        self.sizes = {}
        stream = torch.cuda.current_stream().cuda_stream

        def _alloc(nbytes, user):
            if self.used + nbytes > self.budget:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
            self.used += nbytes
            self.sizes[p] = nbytes
            return p

        def _free(p, user):
            self.used -= self.sizes.pop(p, 0)
            torch.cuda.caching_allocator_delete(p)

        self.alloc = gbpic.ALLOC_FN(_alloc)
        self.free = gbpic.FREE_FN(_free)


@pytest.mark.parametrize("prec", [0, 1])
def test_allocator_exhaustion_is_reported_as_oom(prec):
    """An allocator callback that returns NULL: pic_init_grid fails with PIC_ERR_OOM when
    the grid does not fit, and pic_load_species fails with PIC_ERR_OOM (the reason in
    pic_last_error) when the particles do not; the context stays usable without them."""
    from paper_2609_16575_gb300 import gbpic

    wl = W.thermal((16, 16, 16), 0.2, 8, 0.1, seed=77)
    with pytest.raises(gbpic.PicError) as e:
        gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, allocator=_BudgetAllocator(1 << 10))
    assert e.value.status == gbpic.PIC_ERR_OOM
    budget = _BudgetAllocator(8 << 20)   # the fields fit, the particle blocks do not
    ctx = gbpic.Context(wl.n, wl.d, wl.dt, precision=prec, rho_ion=1.0, allocator=budget)
    with pytest.raises(gbpic.PicError) as e:
        ctx.load_species_array(-1.0, 1.0, wl.species[0].P)
    assert e.value.status == gbpic.PIC_ERR_OOM
    assert b"allocation" in gbpic.lib().pic_last_error(ctx.ptr)
    ctx.step(2)                          # fields only
    ctx.sync()
    assert ctx.diagnostics()["n_alive"] == 0
    ctx.close()


def test_non_finite_field_shows_in_the_maxima():
    """A NaN in E makes the Gauss maxima +inf in pic_diagnostics and in the allocation-free
    check (a max that skipped NaN would report a small residual for a run that blew up)."""
    import ctypes

    from paper_2609_16575_gb300 import gbpic

    n = (16, 8, 8)
    d = (0.2, 0.2, 0.2)
    E = np.zeros((3, n[2], n[1], n[0]))
    E[0, 3, 4, 5] = np.nan
    ctx = gbpic.Context(n, d, W.courant_dt(d, 0.5), precision=0, rho_ion=1.0)
    ctx.set_fields(E, None)
    diag = ctx.diagnostics()
    assert diag["gauss_max"] == np.inf and diag["rho_max"] == 1.0
    g, r = ctypes.c_double(), ctypes.c_double()
    assert gbpic.lib().pic_gauss_check_static(ctx.ptr, ctypes.byref(g), ctypes.byref(r)) == 0
    assert g.value == np.inf and r.value == 1.0
    ctx.close()
