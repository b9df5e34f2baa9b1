"""Host-side contract of bench.py, checked without a GPU: the pair-kernel
source hash that guards the committed ncu traffic figure, the rank
reduction without a process group, and the reference arm's rank rule."""
import os
import shutil
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ("tc_pairs.cu", "tc_epilogue.cuh", "pcc_ptx.cuh", "pcc_sched.h")


def _copy_sources(tmp_path):
    d = tmp_path / "paper_1605_01584_gb300" / "csrc"
    d.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(ROOT, "paper_1605_01584_gb300", "csrc", f),
                    d / f)
    return d


def test_kernel_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    d = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    src = (d / "tc_pairs.cu").read_text()
    (d / "tc_pairs.cu").write_text(
        "// a new comment line\n/* and a block\n   comment */\n" +
        src.replace("namespace pcc {", "namespace pcc {  // trailing", 1))
    assert bench.kernel_source_hash() == h0
    (d / "tc_pairs.cu").write_text(src.replace("kBM = 128", "kBM = 64", 1))
    assert bench.kernel_source_hash() != h0


def test_max_over_ranks_without_group():
    assert bench.max_over_ranks(2.5) == 2.5


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "3",
                        "--warmup", "3"], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
