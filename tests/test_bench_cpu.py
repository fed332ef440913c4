"""Host logic of bench.py: the algorithmic bytes of the streaming model, the
source hash that keys the committed ncu figures to the sources a kernel is
built from, and the roofline line (instruction issue for the frame-resident
kernels, HBM for the streaming ones)."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402
from paper_cs_0609090_gb300 import inputs as I  # noqa: E402


def test_algorithmic_bytes_streaming_model():
    """2 b_z N + 2 S_L per frame-iteration: the qc_n7493 and irr_n64800 figures
    (Section V: S_L = (ceil(d_c/8) + 3) M; per-edge: S_L = E), plus the I/O."""
    w = I.make_workload("qc_n7493", n_frames=2, with_llr=False)
    assert bench.algorithmic_bytes(w.code, "ss_1bit", 30, 1)["per_frame_iter"] == 60452
    assert bench.algorithmic_bytes(w.code, "ss_fixed", 30, 1)["per_frame_iter"] == 116586
    w = I.make_workload("irr_n64800", n_frames=2, with_llr=False)
    b = bench.algorithmic_bytes(w.code, "ss_1bit", 50, 1024)
    assert b["per_frame_iter"] == 518400
    assert b["per_frame_io"] == 64800 + 8100 + 5
    assert b["per_launch"] == 1024 * (50 * 518400 + 64800 + 8100 + 5)
    assert bench.algorithmic_bytes(w.code, "ss_1bit", 50, 1, "f32")["per_frame_iter"] == 1166400


def test_source_hash_follows_the_translation_unit(tmp_path, monkeypatch):
    """The hash covers the code of the kernel's .cu file and of every header it
    includes (transitively), and nothing else."""
    csrc = tmp_path / "paper_cs_0609090_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("int a;\n")
    (csrc / "b.h").write_text('#include "a.cuh"\n')
    (csrc / "k.cu").write_text('#include "b.h"\n// kernel\n')
    (csrc / "other.cu").write_text("int unrelated;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "k_kernel", "k.cu")
    h0 = bench.kernel_source_hash("k_kernel")
    (csrc / "other.cu").write_text("int changed;\n")
    assert bench.kernel_source_hash("k_kernel") == h0
    (csrc / "a.cuh").write_text("int a2;\n")
    h1 = bench.kernel_source_hash("k_kernel")
    assert h1 != h0
    (csrc / "k.cu").write_text('#include "b.h"\nint x = 1;\n')
    h2 = bench.kernel_source_hash("k_kernel")
    assert h2 not in (h0, h1)
    # comments and layout are not code: editing them keeps the hash
    (csrc / "k.cu").write_text('#include "b.h"  // the header\n/* a\n block */ int   x =\n 1;\n')
    assert bench.kernel_source_hash("k_kernel") == h2
    (csrc / "k.cu").write_text('#include "b.h"\nint x = 2;\n')
    assert bench.kernel_source_hash("k_kernel") != h2


def test_code_text_keeps_literals():
    src = 'char* s = "a // b /* c */"; char q = \'\\\'\'; // gone\nint y; /* gone */ int z;'
    assert bench.code_text(src) == 'char* s = "a // b /* c */"; char q = \'\\\'\'; int y; int z;'


def test_committed_figures_are_well_formed():
    """Every entry of profiles/traffic.json names a kernel the bench knows, with a
    positive byte count and a source hash of the bench's form (an entry whose
    sources changed since the capture reads as null, which is not an error)."""
    d = json.load(open(os.path.join(os.path.dirname(HERE), "profiles", "traffic.json")))
    assert d
    for key, e in d.items():
        kernel, workload, form = key.split("/")
        assert kernel in bench.KERNEL_SOURCES, key
        assert workload in I.WORKLOADS and form in ("ss_1bit", "ss_fixed", "two_scan"), key
        assert e["dram_bytes_per_launch"] > 0, key
        assert len(e["source_hash"]) == len(bench.kernel_source_hash(kernel)), key
        assert e.get("warp_inst_per_launch", 1) > 0, key


def test_roofline_line_picks_the_bound():
    w = I.make_workload("qc_n7493", n_frames=2, with_llr=False)
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0}
    r = bench.roofline_line("onchip_h2_kernel", w, "ss_1bit", "int8", 4096, 2.934, clocks, 152)
    if bench.profiled("onchip_h2_kernel", "qc_n7493", "ss_1bit", "warp_inst_per_launch") is None:
        pytest.skip("the kernel's sources changed since its instruction count was captured")
    assert r["bound"] == "alu" and r["unit"] == "G warp-inst/s"
    assert r["peak"] == pytest.approx(152 * 4 * 2.07)
    assert r["achieved"] == pytest.approx(r["warp_inst_per_launch"] / 2.934e-3 / 1e9)
    assert 0.5 < r["frac"] < 1.0
    assert r["hbm_effective"]["frac"] == pytest.approx(
        bench.algorithmic_bytes(w.code, "ss_1bit", 30, 4096)["per_launch"] / 2.934e-3 / 1e9 / r["hbm_effective"]["peak"])
    # no instruction count for this workload/form: the HBM line
    r = bench.roofline_line("onchip_h2_kernel", w, "two_scan", "int8", 4096, 8.4, clocks, 152)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # streaming kernels are HBM lines with their recorded traffic
    w = I.make_workload("irr_n64800", n_frames=2, with_llr=False)
    r = bench.roofline_line("h2s_rows", w, "ss_1bit", "int8", 1024, 14.37, clocks, 152)
    assert r["bound"] == "hbm" and r["algorithmic_bytes_per_launch"] == bench.algorithmic_bytes(
        w.code, "ss_1bit", 50, 1024)["per_launch"]
