"""CPU checks of the C ABI library: it builds, loads, exports every entry point
declared in include/*.h, and validates its arguments (including the CFL bound of
Eq. (15)) before touching a device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2609_16575_gb300 import build, gbpic

    build.build()
    return gbpic.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[\w\*]+\s+)+\**(\w+)\s*\(", src, flags=re.M):
            if m.group(1).startswith("pic"):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for name in sorted(names):
        assert hasattr(L, name), name


def _desc(gbpic, n=(8, 8, 8), d=(0.2, 0.2, 0.2), dt=None):
    desc = gbpic.pic_grid_desc()
    desc.n = (ctypes.c_int32 * 3)(*n)
    desc.d = (ctypes.c_double * 3)(*d)
    desc.dt = dt if dt is not None else 0.5 * 0.2 / 3 ** 0.5
    return desc


def test_argument_validation(L):
    from paper_2609_16575_gb300 import gbpic

    out = ctypes.c_void_p()
    # time step above the CFL limit 1/sqrt(sum 1/d^2)
    bad_dt = _desc(gbpic, dt=1.01 * 0.2 / 3 ** 0.5)
    assert L.pic_init_grid(ctypes.byref(bad_dt), ctypes.byref(out)) == 2          # PIC_ERR_CFL
    assert not out.value
    zero_n = _desc(gbpic, n=(0, 8, 8))
    assert L.pic_init_grid(ctypes.byref(zero_n), ctypes.byref(out)) == 1          # PIC_ERR_ARG
    neg_d = _desc(gbpic, d=(0.2, -0.2, 0.2))
    assert L.pic_init_grid(ctypes.byref(neg_d), ctypes.byref(out)) == 1
    assert L.pic_init_grid(None, ctypes.byref(out)) == 1
    assert L.pic_status_string(2).decode().startswith("time step")
    assert L.pic_step(None, 1) == 1
    assert L.pic_launch_count(None) == 0


def test_no_device_is_reported_not_faked(L):
    """Without a GPU a valid description fails with PIC_ERR_NO_DEVICE: there is no
    CPU fallback behind the ABI."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2609_16575_gb300 import gbpic

    out = ctypes.c_void_p()
    ok = _desc(gbpic)
    assert L.pic_init_grid(ctypes.byref(ok), ctypes.byref(out)) == 10
    assert not out.value


def test_species_descriptor_layout_matches_the_header():
    """The binding's pic_species_desc has the header's fields in the header's order
    (the capacities were appended, so older callers that zero the struct keep working)."""
    from paper_2609_16575_gb300 import gbpic

    src = open(os.path.join(ROOT, "include", "gbpic.h")).read()
    body = src[src.index("typedef struct pic_species_desc {"):src.index("} pic_species_desc;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";")[:-1]:
        decl = decl.replace("typedef struct pic_species_desc {", "").strip()
        declarators = decl.split(None, 1)[1]          # after the type: "x, y" or "*X"
        fields += re.findall(r"\**\s*(\w+)\s*(?:,|$)", declarators)
    assert [f for f, _ in gbpic.pic_species_desc._fields_] == fields


def test_new_entry_points_reject_a_null_context(L):
    """Every setter and the checkpoint calls return PIC_ERR_ARG for a null context (no
    device needed); pic_window_moves reads 0 and pic_free_state accepts NULL."""
    from paper_2609_16575_gb300 import gbpic

    assert L.pic_set_moving_window(None, None) == 1
    assert L.pic_window_moves(None) == 0
    assert L.pic_set_current_filter(None, 1, 1) == 1
    assert L.pic_set_pec(None, 1, 0) == 1
    assert L.pic_set_port(None, None) == 1
    assert L.pic_set_deposit(None, 1) == 1
    assert L.pic_set_shape(None, 2) == 1
    assert L.pic_set_wait_limit(None, 1) == 1
    assert L.pic_probe_fp64_rate(0, None) == 1
    blob, size = ctypes.c_void_p(), ctypes.c_size_t()
    assert L.pic_save_state(None, ctypes.byref(blob), ctypes.byref(size)) == 1
    assert L.pic_load_state(None, None, 0) == 1
    L.pic_free_state(None)
    # the binding mirrors the enumerations of the header
    assert (gbpic.PIC_DEPOSIT_ZIGZAG, gbpic.PIC_DEPOSIT_ESIRKEPOV) == (0, 1)
