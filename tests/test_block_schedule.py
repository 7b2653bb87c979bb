"""Phase-1 schedule of the block iteration kernel, checked on the host.

The kernel stages each tile's two frames in three TMA bands and starts the
products of the first rows before the later bands have landed; with FP32
staging at KR 4 it visits the product rows bottom up so that warps wrapping
from one row to the next stay on distinct shared-memory banks.  A wrong band
threshold would be a race that parity tests can miss, so the helper program
walks the loop pixel by pixel for every storage type, radius and tile shape
(the default and the alternative tile edge) and checks
that no pixel reads a staged row outside the box or of a band not yet waited
for, and that the chosen row order has no more bank conflicts than the other.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_25924_gb300", "csrc")


def test_phase1_band_waits_and_row_order(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "block_schedule_check"
    subprocess.check_call([nvcc, "-std=c++17", "-I", CSRC, "-gencode", "arch=compute_103a,code=sm_103a",
                           os.path.join(HERE, "block_schedule_check.cu"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    assert len(lines) == 76 and lines[-1] == "0 failing cases"
    assert sum(" edge 32 " in l for l in lines) == 3 * 10 and sum(" edge 64 " in l for l in lines) == 3 * 5
    assert sum(" edge 48 NT  512 " in l for l in lines) == 3 * 5  # the persistent kernel's form
    # the FP32 KR 4 tile (the default configuration) runs bottom up, conflict-free
    kr4 = [l for l in lines if l.startswith("f32  KR  4 edge 48 NT  576 ")]
    assert len(kr4) == 1 and "order up" in kr4[0] and " conflicts 0 " in kr4[0]
