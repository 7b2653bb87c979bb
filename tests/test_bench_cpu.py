"""Host-side pieces of bench.py that need no GPU."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = ("k_block.cuh", "k_block_inst.cuh", "iter_math.cuh", "ofv_common.cuh")


def _copy_sources(tmp_path):
    d = tmp_path / "paper_2509_25924_gb300" / "csrc"
    d.mkdir(parents=True)
    for f in CSRC:
        shutil.copy(os.path.join(ROOT, "paper_2509_25924_gb300", "csrc", f), d / f)
    return d


def test_kernel_hash_follows_code_not_comments(tmp_path, monkeypatch):
    """The traffic record of profiles/ is tied to the kernel's code: editing a
    comment keeps the hash, editing a statement changes it."""
    d = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    p = d / "k_block.cuh"
    src = p.read_text()
    p.write_text("// a new comment line\n" + src.replace("// phase 2:", "// phase two:", 1) + "\n/* block\n comment */\n")
    assert bench.kernel_source_hash() == h0
    p.write_text(src.replace("constexpr int kBlockReach = 4;", "constexpr int kBlockReach = 5;", 1))
    assert bench.kernel_source_hash() != h0


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0
