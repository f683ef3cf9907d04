"""CPU checks of bench.py's own arithmetic: the roofline figures, the committed ncu
traffic (used only for the kernel source it was taken on), the FP64 ALU roofline and the
wave fit of the waveguide study."""
import importlib.util
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_arithmetic(bench):
    """achieved = (60 B per particle + 36 B per cell) per launch / average launch time."""
    n_p, n_c = 134217728, 2097152
    kt = {"tile_push": (10, 40.0)}                      # 10 launches, 4 ms each
    r = bench.roofline(kt, "f32", n_p, n_c, 6791.0, "measured", None)
    algo = 60 * n_p + 36 * n_c
    assert r["algorithmic_bytes_per_launch"] == algo
    assert r["achieved"] == pytest.approx(algo / 4e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6791.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["avg_launch_ms"] == pytest.approx(4.0)


def test_committed_traffic_follows_the_kernel_source(bench):
    """The committed ncu traffic is used for the source it was taken on and for no other."""
    with open(os.path.join(ROOT, "profiles", "tile_push_thermal128.json")) as f:
        prof = json.load(f)
    t = bench.committed_traffic("tile_push", "thermal128", 1000)
    if prof["source_sha"] == bench.kernel_source_hash():
        assert t == pytest.approx(prof["dram_bytes_per_particle"] * 1000)
    else:
        assert t is None
    assert bench.committed_traffic("tile_push", "no_such_workload", 1000) is None
    # bytes per particle near the algorithmic 60.6 B: above it (re-reads), but within 2x
    assert 60.6 < prof["dram_bytes_per_particle"] < 121


def test_fp64_alu_roofline(bench):
    kt = {"tile_push": (2, 100.0)}
    r = bench.fp64_alu_roofline(kt, 1_000_000)
    assert r["achieved"] == pytest.approx(bench.FP64_OPS_PER_PARTICLE * 1e6 / 0.05 / 1e12)
    assert r["peak"] == pytest.approx(2 * 152 * 2.07e9 * 2 / 1e12)
    assert r["bound"] == "alu"


def test_wave_fit_recovers_amplitude_and_wave_number(bench):
    x = np.linspace(0.5, 6.5, 700)
    for amp, beta, phi in ((1.0, 5.2397, 0.3), (0.73, 5.2101, -1.2)):
        A, b = bench._fit_wave(x, amp * np.sin(beta * x - phi), 5.22)
        assert A == pytest.approx(amp, rel=1e-9)
        assert b == pytest.approx(beta, rel=1e-9)


def test_host_memory_and_cores_are_positive(bench):
    """The end-to-end leg's host-memory check and the oracle baseline's core count."""
    assert bench.host_memory_available() > 0
    assert bench.host_cores() >= 1


def test_kernel_source_hash_ignores_comments_but_not_code(bench, tmp_path):
    """The hash that guards the committed traffic figures: a comment or layout edit of the
    tile kernel's sources keeps it, any code edit (a string literal included) changes it,
    and the committed traffic files carry the hash of the current source."""
    csrc = tmp_path / "paper_2609_16575_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = {n: open(os.path.join(ROOT, "paper_2609_16575_gb300", "csrc", n)).read()
           for n in ("push.cu", "push_common.cuh", "pic_internal.cuh")}

    def hash_of(files):
        for n, t in files.items():
            (csrc / n).write_text(t)
        return bench.kernel_source_hash(str(tmp_path))

    h0 = hash_of(src)
    assert h0 == bench.kernel_source_hash()
    edited = dict(src, **{"push.cu": "// a new comment line\n" + src["push.cu"].replace("\n", "\n\n", 3) +
                          "\n/* a block\n   comment */\n"})
    assert hash_of(edited) == h0
    assert hash_of(dict(src, **{"push.cu": src["push.cu"] + "\nint extra_symbol;\n"})) != h0
    assert hash_of(dict(src, **{"pic_internal.cuh": src["pic_internal.cuh"].replace('"', '" ', 1)})) != h0
    for name in ("tile_push_stress256.json", "tile_push_thermal128.json"):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            assert json.load(f)["source_sha"] == h0
