"""Host-side contract of bench.py, checked without a GPU: the pair-kernel
source hash that guards the committed ncu traffic figure, the rank
reduction without a process group, the reference arm's rank rule, and that
the reference arm reports the step time it measured."""
import json
import os
import time
import shutil
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ("tc_pairs.cu", "tc_epilogue.cuh", "tc_common.cuh", "pcc_ptx.cuh",
         "pcc_sched.h")


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


def test_reference_arm_reports_measured_steps():
    """ms_per_step is the measured time of one oracle batch: steps x
    ms_per_step fits inside the process's own wall time, and the value is
    the batch's pair*samples over that time."""
    t0 = time.time()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--steps", "3", "--warmup",
                        "1", "--ref-seconds", "2"], capture_output=True,
                       text=True, cwd=ROOT, timeout=600)
    wall = time.time() - t0
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["steps"] == 3
    assert d["steps"] * d["ms_per_step"] / 1e3 < wall
    v = d["pairs_per_step"] * 512 / (d["ms_per_step"] / 1e3) / 1e9
    assert abs(v - d["value"]) <= 1e-9 * v
    assert d["cpu_baseline"]["value"] == d["value"]
