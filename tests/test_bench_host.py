"""Host-side logic of bench.py (no GPU): the clock record, the peak, the
hash that ties a stored ncu traffic figure to the kernel source, and the
traffic file gate."""
import os
import shutil

import pytest

import bench

CSRC = ("paper_1303_4916_gb300", "csrc")


def test_clock_summary_reads_median_max_and_active_reasons():
    lines = [
        "0, 2070, 2070, 250.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 610.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 400.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = bench.ClockSampler.summarize(lines)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    assert r["power_w_max"] == 610.5
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None


def test_fp64_peak_is_two_fma_per_sm_per_clock():
    assert abs(bench.fp64_alu_peak(152, 2070.0) - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-12


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    """A copy of the three kernel source files the hash reads, with bench.ROOT
    pointed at it."""
    dst = tmp_path.joinpath(*CSRC)
    dst.mkdir(parents=True)
    for f in ("eri.cuh", "eri_classes.cuh", "hf_device.h"):
        shutil.copy(os.path.join(bench.ROOT, *CSRC, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def test_kernel_hash_ignores_comments_and_other_kernels(tree):
    h0 = bench.kernel_hash()
    eri = tree / "eri.cuh"
    src = eri.read_text()
    eri.write_text(src.replace("#pragma once", "#pragma once\n// a new comment\n\n", 1))
    assert bench.kernel_hash() == h0
    # the cooperative kernel's section is not part of the dominant kernel
    marker = "// ------------------------------------------------------------- cooperative kernel\n"
    eri.write_text(src.replace(marker, marker + "static const int unrelated_probe = 1;\n", 1))
    assert bench.kernel_hash() == h0
    # code of the (ps|ss) class changes the hash
    gen = tree / "eri_classes.cuh"
    g = gen.read_text()
    i = g.index("struct C_ps_ss {")
    gen.write_text(g[:i] + g[i:].replace("B[1]", "B[0]", 1))
    assert bench.kernel_hash() != h0


def test_traffic_is_reported_only_for_matching_source(tree):
    prof = os.path.join(bench.ROOT, "profiles", "eri_jk_c2_traffic.txt")
    with open(prof, "w") as fh:
        fh.write(f"# comment\nclass=(ps|ss)\nkernel_hash={bench.kernel_hash()}\ndram_bytes_per_launch=1234\n")
    assert bench.ncu_traffic("(ps|ss)") == 1234.0
    assert bench.ncu_traffic("(ps|ps)") is None
    with open(prof, "w") as fh:
        fh.write("class=(ps|ss)\nkernel_hash=0000000000000000\ndram_bytes_per_launch=1234\n")
    assert bench.ncu_traffic("(ps|ss)") is None
