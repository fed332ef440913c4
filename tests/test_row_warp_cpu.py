"""The warp -> (frame chunk, checks) mappings of the streaming row kernels,
compiled from their header with g++ and checked on the CPU: one-to-one over the
launched grid for every chunk interleave, including chunk counts that the
interleave does not divide (a last, partial chunk group)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_cs_0609090_gb300", "csrc")


def test_row_warp_covers_every_chunk_and_check_once(tmp_path):
    exe = str(tmp_path / "row_warp_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "row_warp_check.cpp"), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]
    assert r.stdout.strip().endswith("0 of 1368 cases fail"), r.stdout[-500:]
